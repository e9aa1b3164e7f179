"""GPU <-> oracle parity of the CUDA path, called through the C ABI.

Tolerance: 1e-12 relative max-norm per step (1e-9 after 100 steps), the
parity bar of the FP64 path; per-kernel residuals are held to the same
1e-12 relative to the largest residual entry.
"""
import numpy as np
import pytest

from oracle import Oracle
from paper_2609_10849_b300 import workloads
from tests.test_oracle_hydro import smooth_random_state
from tests.test_oracle_magnetic import random_mag_state
from tests.util import oracle_state

pytestmark = pytest.mark.gpu

PK = [(1, 0), (1, 1), (2, 1), (2, 2), (3, 2), (3, 3), (4, 3), (4, 4)]


def rel(a, b, floor=0.0):
    """max|a - b| / max(max|b|, floor): relative max-norm; the floor is the
    scale of the quantity where the field itself is zero up to roundoff."""
    a, b = np.asarray(a), np.asarray(b)
    den = max(np.abs(b).max(), floor)
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


def solver_like(o):
    from paper_2609_10849_b300.mhd import Solver
    return Solver(o.nx, o.ny, o.p, o.m, o.gamma, o.domain)


def copy_state(o, s):
    s.set_state(*o.get_state())


def compare_state(o, s, tol):
    Uo, Bxo, Byo, Bzo = o.get_state()
    Ug, Bxg, Byg, Bzg = s.get_state()
    bscale = max(np.abs(Bxo).max(), np.abs(Byo).max(), np.abs(Bzo).max())
    errs = [rel(Ug[c], Uo[c], np.abs(Uo).max()) for c in range(5)] + \
        [rel(Bxg, Bxo, bscale), rel(Byg, Byo, bscale), rel(Bzg, Bzo, bscale)]
    # max() over a list holding a NaN need not return the NaN: test finiteness first
    assert all(np.isfinite(a).all() for a in (Uo, Bxo, Byo, Bzo, Ug, Bxg, Byg, Bzg)), "non-finite state"
    assert max(errs) <= tol, errs
    return max(errs)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("mesh", [(5, 4), (7, 3), (1, 1), (2, 1)])
def test_hydro_rhs(p, mesh):
    rng = np.random.default_rng(p * 10 + mesh[0])
    o = Oracle(*mesh, p, p, 1.4, (0.0, 1.0, 0.0, 0.8))
    U = smooth_random_state(o, rng)
    Lo = o.hydro_rhs(U)
    s = solver_like(o)
    Lg = s.hydro_rhs(U.copy())
    # floor: the residual scale max|U| (p+1)^2 / h; on a single periodic element
    # at p = 1 the state is a free stream and the residual itself is roundoff
    floor = 1e-3 * np.abs(U).max() * (p + 1) ** 2 / min(1.0 / mesh[0], 0.8 / mesh[1])
    for c in range(5):
        assert rel(Lg[c], Lo[c], floor) <= 1e-12, (c, rel(Lg[c], Lo[c], floor))


@pytest.mark.parametrize("pk", PK)
@pytest.mark.parametrize("resistive", [False, True])
def test_mag_rhs(pk, resistive):
    p, k = pk
    rng = np.random.default_rng(100 + 10 * p + k)
    o = Oracle(5, 3, p, k, 5 / 3, (0.0, 1.3, 0.0, 0.7))
    rho, e, u, Bx, By, Bz = random_mag_state(o, rng)
    eta = rng.uniform(0.0, 0.3, o.K) if resistive else np.zeros(o.K)
    eta[::3] = 0.0
    ro = o.mag_rhs(rho, e, u, Bx, By, Bz, eta)
    s = solver_like(o)
    rg = s.mag_rhs(rho, e, u, Bx, By, Bz, eta)
    for key in ("du", "dBx", "dBy", "dBz"):
        assert rel(rg[key], ro[key]) <= 1e-12, (key, rel(rg[key], ro[key]))
    if resistive:
        assert rel(rg["de"], ro["de"]) <= 1e-12
    else:
        assert np.all(rg["de"] == 0.0)


@pytest.mark.parametrize("which", ["H", "M"])
@pytest.mark.parametrize("pk", PK)
def test_substep(which, pk):
    wl = workloads.orszag_tang()
    o = oracle_state(wl, 6, 5, *pk)
    s = solver_like(o)
    copy_state(o, s)
    tau = 0.5 * o.cfl_dt()
    assert o.substep(which, tau) == 0
    s.substep(which, tau)
    compare_state(o, s, 1e-12)


def test_cfl_dt():
    wl = workloads.orszag_tang()
    o = oracle_state(wl, 8, 8, 3, 3)
    s = solver_like(o)
    copy_state(o, s)
    assert s.compute_dt() == pytest.approx(o.cfl_dt(), rel=1e-14)


def test_potential_field_and_coords():
    from paper_2609_10849_b300.mhd import Solver
    wl = workloads.orszag_tang()
    o = oracle_state(wl, 6, 4, 3, 3)
    s = Solver(6, 4, 3, 3, wl["gamma"], wl["domain"])
    for which in ("dg", "w", "bz"):
        Xo, Yo = o.coords(which)
        Xg, Yg = s.coords(which)
        assert np.abs(Xo - Xg).max() < 1e-15 and np.abs(Yo - Yg).max() < 1e-15
    XW, YW = s.coords("w")
    XZ, YZ = s.coords("bz")
    s.set_B_from_potential(wl["Az"](XW, YW), *wl["B0"], wl["fields"](XZ, YZ)[5])
    _, Bxg, Byg, _ = s.get_state()
    _, Bxo, Byo, _ = o.get_state()
    assert rel(Bxg, Bxo) <= 1e-13 and rel(Byg, Byo) <= 1e-13


@pytest.mark.parametrize("pk", PK)
@pytest.mark.parametrize("nq", [None, 16])
def test_bz_projection(pk, nq):
    """Initial B_z as the L2 projection onto V_h^k (reading R10): the GPU's
    tensor-factored projection against the oracle's element normal equations,
    with the Gauss points of both sides."""
    from paper_2609_10849_b300.mhd import Solver
    p, k = pk
    nq = k + 3 if nq is None else nq
    wl = workloads.alfven_diagonal()
    o = oracle_state(wl, 5, 3, p, k)
    s = Solver(5, 3, p, k, wl["gamma"], wl["domain"])
    copy_state(o, s)
    Xo, Yo = o.quad_coords(nq)
    Xg, Yg = s.quad_coords(nq)
    assert np.abs(Xo - Xg).max() < 1e-14 and np.abs(Yo - Yg).max() < 1e-14
    f = np.sin(1.3 * Xg - 0.7) * np.cos(0.9 * Yg) + 0.1 * Xg
    o.project_Bz(f, nq)
    s.set_Bz_projected(f, nq)
    compare_state(o, s, 1e-13)
    import torch  # device input
    s.set_state(*o.get_state())
    s.set_Bz_projected(torch.tensor(2.0 * f, device="cuda"), nq)
    o.project_Bz(2.0 * f, nq)
    compare_state(o, s, 1e-13)


def test_strang_alfven_per_step():
    """Circularly polarised Alfven wave (16 x 16, p = k = 3): 1e-12 per step."""
    wl = workloads.alfven_rotated()
    o = oracle_state(wl, 16, 16, 3, 3)
    o.set_params(cfl=0.4)
    s = solver_like(o)
    copy_state(o, s)
    for _ in range(3):
        dt = o.cfl_dt()
        assert s.compute_dt() == pytest.approx(dt, rel=1e-13)
        o.strang_step(dt)
        s.strang_step(dt)
        compare_state(o, s, 1e-12)
        copy_state(o, s)  # per-step parity from an identical input


def test_strang_alfven_100_steps():
    """The circularly polarised Alfven wave over 100 Strang steps: within 1e-9 of the oracle."""
    wl = workloads.alfven_rotated()
    o = oracle_state(wl, 16, 16, 3, 3)
    s = solver_like(o)
    copy_state(o, s)
    dt = o.cfl_dt()
    for _ in range(100):
        o.strang_step(dt)
    assert s.strang_steps(dt, 100) == 100
    compare_state(o, s, 1e-9)
    d = s.diagnostics()
    do = o.diagnostics()
    assert d["mass"] == pytest.approx(do["mass"], rel=1e-14)
    assert d["div_B"] <= 1e-12 * d["B_max"]


def tiled(o, reps):
    """Host state of the oracle tiled reps x reps times (same element geometry)."""
    U, Bx, By, Bz = o.get_state()
    n2, mm = o.n2, o.mm
    U4 = U.reshape(5, o.ny, o.nx, n2)
    Ut = np.tile(U4, (1, reps, reps, 1)).reshape(5, -1)
    Bzt = np.tile(Bz.reshape(o.ny, o.nx, mm * mm), (reps, reps, 1)).ravel()
    Bxt = np.tile(Bx.reshape(o.ny * mm, o.nx * mm), (reps, reps)).ravel()
    Byt = np.tile(By.reshape(o.ny * mm, o.nx * mm), (reps, reps)).ravel()
    return Ut, Bxt, Byt, Bzt


def test_full_size_tiled_parity():
    """256 x 256 elements (the Orszag-Tang mesh size) in the bench launch
    configuration: a state tiled 16 x 16 from a 16 x 16 oracle state must give
    the oracle's step on every tile."""
    from paper_2609_10849_b300.mhd import Solver
    wl = workloads.orszag_tang()
    o = oracle_state(wl, 16, 16, 3, 3)
    reps = 16
    x0, x1, y0, y1 = o.domain
    s = Solver(16 * reps, 16 * reps, 3, 3, wl["gamma"], (x0, x0 + reps * (x1 - x0), y0, y0 + reps * (y1 - y0)))
    s.set_state(*tiled(o, reps))
    dt = o.cfl_dt()
    assert s.compute_dt() == pytest.approx(dt, rel=1e-13)
    o.strang_step(dt)
    s.strang_step(dt)
    U, Bx, By, Bz = s.get_state()
    Ut, Bxt, Byt, Bzt = tiled(o, reps)
    for a, b in [(U, Ut), (Bx, Bxt), (By, Byt), (Bz, Bzt)]:
        assert rel(a, b) <= 1e-12
    d = s.diagnostics()
    assert d["div_B"] <= 1e-12 * d["B_max"]


STAB = dict(oe_hydro=1, oe_vel=1, pp=1, ar=1, s_H=0.02, s_M=0.02, C_s=5.0, C_eta=0.2)


def stab_pair(wl, nx, ny, p, k, **over):
    prm = dict(STAB, **over)
    o = oracle_state(wl, nx, ny, p, k)
    o.set_params(cfl=0.4, **prm)
    s = solver_like(o)
    s.set_params(cfl=0.4, **prm)
    copy_state(o, s)
    return o, s


@pytest.mark.parametrize("pk", PK)
def test_stabilised_hydro_substep(pk):
    o, s = stab_pair(workloads.orszag_tang(), 8, 6, *pk, oe_vel=0, ar=0)
    tau = 0.5 * o.cfl_dt()
    assert o.substep("H", tau) == 0
    s.substep("H", tau)
    compare_state(o, s, 1e-12)


@pytest.mark.parametrize("pk", PK)
def test_stabilised_magnetic_substep(pk):
    o, s = stab_pair(workloads.orszag_tang(), 8, 6, *pk, oe_hydro=0, pp=0)
    tau = o.cfl_dt()
    assert o.substep("M", tau) == 0
    s.substep("M", tau)
    compare_state(o, s, 1e-12)
    eo, eg = o.eta(), s.eta()
    assert eo.max() > 0
    # eta comes from jumps of nearly equal B traces (J_0 ~ 1e-4 against |B| ~ 0.3),
    # so its roundoff is amplified by |B|/J_0; the state it drives matches at 1e-12
    assert rel(eg, eo) <= 1e-9


def _planar(a):
    """Largest |value| of the out-of-plane fields u_z (momentum) and B_z."""
    U, _, _, Bz = a
    return max(np.abs(U[3]).max(), np.abs(Bz).max())


@pytest.mark.parametrize("pk", [(1, 0), (2, 2), (3, 3)])
def test_uniform_state_is_steady_with_stabilisation(pk):
    """Free stream with every stabilisation map on: every sensor component is
    constant to roundoff (reading R8), so no map may act; the state stays
    finite and uniform and matches the oracle step for step."""
    from paper_2609_10849_b300.mhd import Solver
    p, k = pk
    o = Oracle(6, 5, p, k, 5 / 3, (0.0, 1.0, 0.0, 0.8))
    X, Y = o.coords("dg")
    one = np.ones_like(X)
    u = np.stack([0.3 * one, -0.2 * one, 0.1 * one])
    Bx, By = o.b_from_potential(np.zeros(o.G), 0.5, 0.2)
    o.set_primitive(one, u, one, Bx, By, np.full(o.Z, 0.1))
    o.set_params(cfl=0.4, **STAB)
    s = Solver(6, 5, p, k, 5 / 3, (0.0, 1.0, 0.0, 0.8))
    s.set_params(cfl=0.4, **STAB)
    copy_state(o, s)
    x0 = [a.copy() for a in o.get_state()]
    dt = o.cfl_dt()
    for _ in range(2):
        assert o.strang_step(dt)[0] == 0
        assert s.strang_step(dt)[0] == 0
        compare_state(o, s, 1e-12)
        copy_state(o, s)
    for a, b in zip(s.get_state(), x0):
        assert np.abs(a - b).max() <= 1e-13 * max(np.abs(b).max(), 1.0)
    assert s.diagnostics()["stab_active"] == 0  # no map acted


@pytest.mark.parametrize("pk", PK)
@pytest.mark.parametrize("wl_name", ["orszag_tang", "blast"])
def test_reduced_2d2v_stage(pk, wl_name):
    """The reduced 2D2V magnetic stage (u_z = B_z = 0; in-plane E_h and J_h
    not formed) on 2D2V states, every stabilisation map on (A.R. resistive):
    equal to the full stage to rounding-order zero (the skipped terms are exact
    zeros), against the oracle's full stage at 1e-12, and u_z, B_z stay 0."""
    wl = workloads.WORKLOADS[wl_name]()
    o, s = stab_pair(wl, 8, 6, *pk)
    f = solver_like(o)
    f.set_params(cfl=0.4, **STAB)
    copy_state(o, f)
    s.set_params(reduced_2d2v=1)
    assert _planar(s.get_state()) == 0.0
    tau = o.cfl_dt()
    assert o.substep("M", tau) == 0
    s.substep("M", tau)
    f.substep("M", tau)
    compare_state(o, s, 1e-12)
    for a, b in zip(s.get_state(), f.get_state()):
        assert np.array_equal(a, b)
    assert _planar(s.get_state()) == 0.0
    if wl_name == "orszag_tang":  # the blast's uniform field leaves the A.R. sensor off
        assert s.eta().max() > 0


@pytest.mark.parametrize("pk", [(1, 1), (2, 2), (3, 3), (4, 3)])
def test_reduced_2d2v_strang_steps(pk):
    """Graph-replayed Strang steps with the reduced stage against the full
    stage (bitwise) and the oracle (1e-12 per step)."""
    o, s = stab_pair(workloads.orszag_tang(), 12, 10, *pk)
    f = solver_like(o)
    f.set_params(cfl=0.4, **STAB)
    copy_state(o, f)
    s.set_params(reduced_2d2v=1)
    dt = o.cfl_dt()
    assert s.strang_steps(dt, 3) == 3  # three steps in one graph: bitwise the full stage's
    assert f.strang_steps(dt, 3) == 3
    for a, b in zip(s.get_state(), f.get_state()):
        assert np.array_equal(a, b)
    assert _planar(s.get_state()) == 0.0
    copy_state(o, s)
    for _ in range(3):  # per step against the oracle from identical inputs
        st_o, _, _ = o.strang_step(dt)
        assert st_o == 0
        assert s.strang_steps(dt, 1) == 1
        compare_state(o, s, 1e-12)
        copy_state(o, s)


@pytest.mark.parametrize("wl_name", ["orszag_tang", "blast"])
@pytest.mark.parametrize("pk", [(1, 1), (2, 1), (3, 3)])
def test_stabilised_strang_steps(wl_name, pk):
    """The benchmark and blast physics on small meshes, all stabilisation on, per-step parity from identical inputs."""
    wl = workloads.WORKLOADS[wl_name]()
    o, s = stab_pair(wl, 12, 12, *pk)
    for _ in range(3):
        dt = o.cfl_dt()
        st_o, taken_o, _ = o.strang_step(dt)
        st_g, taken_g = s.strang_step(dt)
        assert st_o in (0, 1) and taken_g == taken_o
        compare_state(o, s, 1e-12)
        copy_state(o, s)
    d = s.diagnostics()
    assert d["rho_min"] > 0 and d["p_min"] > 0
    assert d["div_B"] <= 1e-12 * d["B_max"]


def test_full_size_tiled_parity_stabilised():
    """The benchmark configuration (256 x 256, p = k = 3, OE + PP + A.R. + velocity
    filter): tiling a 16 x 16 oracle state 16 x 16 times keeps every row, column
    and global statistic of the sensors, so each tile must reproduce the
    oracle's stabilised Strang step."""
    from paper_2609_10849_b300.mhd import Solver
    wl = workloads.orszag_tang()
    o = oracle_state(wl, 16, 16, 3, 3)
    o.set_params(cfl=0.4, **STAB)
    reps = 16
    x0, x1, y0, y1 = o.domain
    s = Solver(16 * reps, 16 * reps, 3, 3, wl["gamma"], (x0, x0 + reps * (x1 - x0), y0, y0 + reps * (y1 - y0)))
    s.set_params(cfl=0.4, **STAB)
    s.set_state(*tiled(o, reps))
    dt = o.cfl_dt()
    o.strang_step(dt)
    s.strang_step(dt)
    U, Bx, By, Bz = s.get_state()
    Ut, Bxt, Byt, Bzt = tiled(o, reps)
    bscale = max(np.abs(Bxt).max(), np.abs(Byt).max())
    assert rel(U, Ut) <= 1e-12
    for a, b in [(Bx, Bxt), (By, Byt), (Bz, Bzt)]:
        assert rel(a, b, bscale) <= 1e-12
    eta_t = np.tile(o.eta().reshape(16, 16), (reps, reps)).ravel()
    assert rel(s.eta(), eta_t) <= 1e-9


def test_full_size_blast_1024_tiled():
    """The blast wave at its full size (1024 x 1024 elements, p = k = 3, every
    stabilisation map on, in the bench's launch configuration): a 64 x 64 blast
    tiled 16 x 16 times keeps every row, column and global sensor statistic,
    so every tile must reproduce the oracle's stabilised Strang step; mass is
    conserved and B stays divergence-free at this size."""
    from paper_2609_10849_b300.mhd import Solver
    wl = workloads.blast()
    o = oracle_state(wl, 64, 64, 3, 3)
    o.set_params(cfl=0.4, **STAB)
    reps = 16
    x0, x1, y0, y1 = o.domain
    s = Solver(64 * reps, 64 * reps, 3, 3, wl["gamma"], (x0, x0 + reps * (x1 - x0), y0, y0 + reps * (y1 - y0)))
    s.set_params(cfl=0.4, **STAB)
    s.set_state(*tiled(o, reps))
    d0 = s.diagnostics()
    dt = o.cfl_dt()
    assert o.strang_step(dt)[0] == 0
    st, taken = s.strang_step(dt)
    assert st == 0 and taken == dt
    U, Bx, By, Bz = s.get_state()
    Ut, Bxt, Byt, Bzt = tiled(o, reps)
    bscale = max(np.abs(Bxt).max(), np.abs(Byt).max())
    assert rel(U, Ut) <= 1e-12
    for a, b in [(Bx, Bxt), (By, Byt), (Bz, Bzt)]:
        assert rel(a, b, bscale) <= 1e-12
    d1 = s.diagnostics()
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert d1["div_B"] <= 1e-12 * d1["B_max"]
    assert d1["rho_min"] > 0 and d1["p_min"] > 0


def test_diagnostics_activity_and_rejections():
    """stab_active reports the maps that acted since the previous diagnostics
    call (and is cleared by reading it); n_rejections counts retried attempts."""
    wl = workloads.blast()
    o = oracle_state(wl, 16, 16, 3, 3)
    s = solver_like(o)
    s.set_params(cfl=0.4, **STAB)
    copy_state(o, s)
    assert s.diagnostics()["stab_active"] == 0
    dt = o.cfl_dt()
    for _ in range(2):
        assert s.strang_step(dt)[0] == 0
    d = s.diagnostics()
    assert d["stab_active"] & 1  # the hydro OE damps the blast's jump
    assert d["n_rejections"] == 0
    assert s.diagnostics()["stab_active"] == 0
    st, taken = s.strang_step(200 * dt)  # far beyond the CFL step: rejected and halved
    assert st == 1 and taken < 200 * dt
    assert s.diagnostics()["n_rejections"] >= 1


@pytest.mark.parametrize("pk", [(1, 1), (2, 2), (3, 3), (4, 4)])
def test_strang_mhm_order_parity(pk):
    """The M-H-M composition (reading R20), every stabilisation map on: per-step
    parity with the oracle's M-H-M step."""
    o, s = stab_pair(workloads.orszag_tang(), 8, 8, *pk)
    o.set_strang_order(1)
    s.set_params(strang_order=1)
    for _ in range(2):
        dt = o.cfl_dt()
        st_o, taken_o, _ = o.strang_step(dt)
        st_g, taken_g = s.strang_step(dt)
        assert st_o == 0 and st_g == 0 and taken_g == taken_o
        compare_state(o, s, 1e-12)
        copy_state(o, s)
