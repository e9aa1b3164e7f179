"""GPU <-> oracle parity of the branches of the stabilisation and of the step
driver that smooth workloads do not reach, through the C ABI:

* the positivity limiter's edge cases (reading R9) on hand-built elements,
  through the stage-map test hook: vacuum collapse to the element average,
  the density scaling landing on the floor 64 eps, the pressure scaling, and
  the collapse of an element whose average pressure is below eps_p;
* a Strang step on a cold double rarefaction, where the limiter provably acts
  (without it the oracle rejects the same step nine times);
* rejection and retry (reading R3): status, dt taken, rejection count and
  state against the oracle; halvings exhausted (MHD_INADMISSIBLE) with the
  state restored bit for bit;
* every diagnostics field against the oracle's;
* meshes one element wide (periodic self-neighbours in the closures);
* the library's refined FP64 reciprocal against IEEE division.

Tolerance: 1e-12 relative max-norm, as for the other parity tests; per node
relative to the element's own scale where elements differ by many orders of
magnitude (a collapsed near-vacuum element next to unit states).
"""
import math

import numpy as np
import pytest

from oracle import INADMISSIBLE, Oracle
from paper_2609_10849_b300 import workloads
from tests.test_gpu_parity import PK, compare_state, copy_state, rel, solver_like, stab_pair
from tests.test_oracle_magnetic import random_mag_state
from tests.test_oracle_stab import EPS, _uniform_state, elem_avg
from tests.util import oracle_state

pytestmark = pytest.mark.gpu

STAB = dict(oe_hydro=1, oe_vel=1, pp=1, ar=1, s_H=0.02, s_M=0.02, C_s=5.0, C_eta=0.2)


def _per_element_close(o, a, b, tol=1e-12):
    """|a - b| <= tol * (largest |b| of the element's component) node by node."""
    A = a.reshape(5, o.K, o.n2)
    B = b.reshape(5, o.K, o.n2)
    scale = np.abs(B).max(axis=2, keepdims=True)
    scale = np.where(scale > 0, scale, 1e-300)
    err = (np.abs(A - B) / scale).max()
    assert np.isfinite(A).all() and err <= tol, err
    return err


def _vacuum(rng):
    o = Oracle(3, 2, 2, 2, 1.4)
    U = _uniform_state(o)
    sl = slice(4 * o.n2, 5 * o.n2)
    U[:, sl] *= 1e-17  # average density 1e-17 < 64 eps: collapse
    U[0, sl] *= 1.0 + 0.5 * rng.uniform(-1, 1, o.n2)
    return o, U, [4]


def _density_floor(rng):
    o = Oracle(2, 2, 3, 3, 1.4)
    U = _uniform_state(o)
    sl = slice(1 * o.n2, 2 * o.n2)
    rho = np.linspace(1.5, 0.5, o.n2)
    rho[3] = -0.2  # one negative node, positive average: scaled onto the floor
    U[0, sl] = rho
    U[1:4, sl] = 0.0
    U[4, sl] = 5.0
    return o, U, [1]


def _pressure_scaling(rng):
    o = Oracle(3, 2, 3, 3, 1.4)
    U = _uniform_state(o, rho=1.0, u=(0.5, 0.2, 0.0), p=0.3)
    sl = slice(2 * o.n2, 3 * o.n2)
    U[0, sl] *= 1.0 + 0.2 * rng.uniform(-1, 1, o.n2)
    kin = 0.5 * (U[1, sl] ** 2 + U[2, sl] ** 2 + U[3, sl] ** 2) / U[0, sl]
    U[4, sl] = kin + 0.3 / 0.4
    U[4, 2 * o.n2 + 5] = kin[5] - 0.2  # one node with negative pressure, positive average
    return o, U, [2]


def _pressure_collapse(rng):
    o = Oracle(2, 3, 2, 2, 1.4)
    U = _uniform_state(o)
    sl = slice(3 * o.n2, 4 * o.n2)
    U[0, sl] = 1.0 + 0.3 * rng.uniform(-1, 1, o.n2)
    U[1, sl] = U[0, sl] * 1.0
    U[2:4, sl] = 0.0
    # average pressure 0.4 * 1e-12 * ~0.5, below eps_p = 8192 eps S ~ 1.8e-12
    U[4, sl] = 0.5 * U[1, sl] ** 2 / U[0, sl] * (1.0 + 1e-12)
    return o, U, [3]


CASES = {"vacuum_collapse": _vacuum, "density_floor": _density_floor, "pressure_scaling": _pressure_scaling,
         "pressure_collapse": _pressure_collapse}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("oe", [0, 1])
def test_limiter_edge_cases_match_the_oracle(case, oe):
    rng = np.random.default_rng(11)
    o, U, limited = CASES[case](rng)
    tau = 1e-6 if oe else 0.0  # with the OE: a short stage, so its damping leaves the edge in place
    o.set_params(pp=1, oe_hydro=oe, s_H=0.02)
    want = o.hydro_stage_map(U, tau)
    s = solver_like(o)
    s.set_params(pp=1, oe_hydro=oe, s_H=0.02)
    z = np.zeros(o.G)
    s.set_state(_uniform_state(o), z, z, np.zeros(o.Z))
    s.diagnostics()  # clear the activity word
    got = s.hydro_stage_map(U, tau)
    _per_element_close(o, got, want)
    assert s.diagnostics()["stab_active"] & 2  # the limiter acted
    # the edge itself: the averages are kept, and the limited elements obey
    # the branch's outcome
    np.testing.assert_allclose(elem_avg(o, got), elem_avg(o, U), rtol=1e-12, atol=1e-30)
    G = got.reshape(5, o.K, o.n2)
    for k in limited:
        if case in ("vacuum_collapse", "pressure_collapse"):
            assert np.all(G[:, k] == G[:, k, :1])
        elif case == "density_floor":
            assert abs(G[0, k].min() - 64 * EPS) <= 1e-12
        else:  # scaled towards the average: every nodal pressure positive now
            pr = 0.4 * (G[4, k] - 0.5 * (G[1, k] ** 2 + G[2, k] ** 2 + G[3, k] ** 2) / G[0, k])
            Uk = U.reshape(5, o.K, o.n2)[:, k]
            pr0 = 0.4 * (Uk[4] - 0.5 * (Uk[1] ** 2 + Uk[2] ** 2 + Uk[3] ** 2) / Uk[0])
            assert pr0.min() < 0.0 < pr.min()


def _cold_rarefaction(p, k, pp):
    """rho = 1, p = 1e-3, u_x = -2 for x < 1/2 and +2 beyond (a cold double
    rarefaction with a collision at the periodic seam)."""
    o = Oracle(16, 2, p, k, 1.4, (0.0, 1.0, 0.0, 0.25))
    X, _ = o.coords("dg")
    u = np.stack([np.where(X < 0.5, -2.0, 2.0), 0 * X, 0 * X])
    Bx, By = o.b_from_potential(np.zeros(o.G), 0.0, 0.0)
    o.set_primitive(np.ones_like(X), u, np.full_like(X, 1e-3), Bx, By, np.zeros(o.Z))
    o.set_params(oe_hydro=1, pp=pp, cfl=0.4)
    return o


@pytest.mark.parametrize("pk", [(2, 2), (3, 3)])
def test_strang_step_where_the_limiter_acts(pk):
    o = _cold_rarefaction(*pk, pp=1)
    s = solver_like(o)
    s.set_params(oe_hydro=1, pp=1, cfl=0.4)
    copy_state(o, s)
    probe = _cold_rarefaction(*pk, pp=0)
    dt = o.cfl_dt()
    st_probe, _, nrej = probe.strang_step(dt)
    assert nrej >= 1  # without the limiter the same step is rejected
    s.diagnostics()
    for _ in range(2):
        st_o, taken_o, nrej_o = o.strang_step(dt)
        st_g, taken_g = s.strang_step(dt)
        assert st_o == 0 and nrej_o == 0 and st_g == 0 and taken_g == taken_o
        compare_state(o, s, 1e-12)
        assert s.diagnostics()["stab_active"] & 2
        copy_state(o, s)


@pytest.mark.parametrize("pk", [(2, 2), (3, 3)])
def test_rejection_and_retry_match_the_oracle(pk):
    """Without the limiter the cold rarefaction's CFL step has inadmissible raw
    averages: both sides halve dt the same number of times (reading R3)."""
    o = _cold_rarefaction(*pk, pp=0)
    s = solver_like(o)
    s.set_params(oe_hydro=1, pp=0, cfl=0.4)
    copy_state(o, s)
    n0 = s.diagnostics()["n_rejections"]
    dt = o.cfl_dt()
    st_o, taken_o, nrej_o = o.strang_step(dt)
    st_g, taken_g = s.strang_step(dt)
    assert nrej_o >= 1 and st_o == 1
    assert st_g == 1 and taken_g == taken_o == dt * 0.5 ** nrej_o
    assert s.diagnostics()["n_rejections"] - n0 == nrej_o
    compare_state(o, s, 1e-12)


def test_halvings_exhausted_restore_the_state():
    """A negative element-average density is inadmissible for every halving:
    after max_halvings = 3 both sides report it, count 4 rejections and
    restore the state bit for bit."""
    from paper_2609_10849_b300.mhd import MHD_INADMISSIBLE, MhdError
    o = Oracle(3, 3, 2, 2, 1.4)
    o.set_params(pp=1, max_halvings=3)
    U = _uniform_state(o)
    U[0, 2 * o.n2:3 * o.n2] = -0.5
    z = np.zeros(o.G)
    o.set_state(U, z, z, np.zeros(o.Z))
    s = solver_like(o)
    s.set_params(pp=1, max_halvings=3)
    copy_state(o, s)
    before = [a.copy() for a in s.get_state()]
    st, _, nrej = o.strang_step(1e-3)
    assert st == INADMISSIBLE and nrej == 4
    with pytest.raises(MhdError) as e:
        s.strang_step(1e-3)
    assert e.value.code == MHD_INADMISSIBLE
    assert s.diagnostics()["n_rejections"] == 4
    for a, b in zip(s.get_state(), before):
        assert np.array_equal(a, b)


def _diag_compare(o, s):
    do, dg = o.diagnostics(), s.diagnostics()
    escale = do["E_kin"] + do["E_int"] + do["E_mag"]
    mscale = math.sqrt(2.0 * do["mass"] * (do["E_kin"] + do["E_int"]))
    for key in ("mass", "E_kin", "E_int", "E_mag"):
        assert abs(dg[key] - do[key]) <= 1e-12 * abs(do[key]), key
    for key in ("mom_x", "mom_y", "mom_z"):
        assert abs(dg[key] - do[key]) <= 1e-12 * mscale, key
    assert abs(dg["entropy"] - do["entropy"]) <= 1e-12 * max(abs(do["entropy"]), escale), "entropy"
    assert dg["rho_min"] == do["rho_min"]
    assert abs(dg["p_min"] - do["p_min"]) <= 1e-13 * do["p_min"]
    assert abs(dg["B_max"] - do["B_max"]) <= 1e-13 * do["B_max"]
    assert dg["div_B"] <= 1e-12 * dg["B_max"] and do["div_B"] <= 1e-12 * do["B_max"]
    assert abs(dg["eta_max"] - do["eta_max"]) <= 1e-9 * max(do["eta_max"], 1e-300)
    return do, dg


@pytest.mark.parametrize("wl_name", ["orszag_tang", "blast"])
@pytest.mark.parametrize("pk", [(2, 2), (3, 3)])
def test_every_diagnostics_field_matches_the_oracle(wl_name, pk):
    wl = workloads.WORKLOADS[wl_name]()
    o, s = stab_pair(wl, 10, 8, *pk)
    _diag_compare(o, s)
    dt = o.cfl_dt()
    for _ in range(2):
        assert o.strang_step(dt)[0] == 0
        s.strang_step(dt)
        copy_state(o, s)  # identical states: the diagnostics themselves are compared
        do, dg = _diag_compare(o, s)
    if wl_name == "orszag_tang":
        assert do["eta_max"] > 0


@pytest.mark.parametrize("mesh", [(1, 1), (1, 3), (3, 1)])
@pytest.mark.parametrize("pk", [(1, 0), (2, 2), (3, 2), (4, 4)])
def test_one_element_wide_meshes_magnetic_residual(mesh, pk):
    """An element is its own periodic neighbour across a direction one
    element wide: the closures and the assembly over shared DOFs meet the
    same element on both sides."""
    p, k = pk
    rng = np.random.default_rng(7 * p + k + mesh[0])
    o = Oracle(*mesh, p, k, 5 / 3, (0.0, 0.9, 0.0, 1.1))
    rho, e, u, Bx, By, Bz = random_mag_state(o, rng)
    eta = rng.uniform(0.0, 0.3, o.K)
    ro = o.mag_rhs(rho, e, u, Bx, By, Bz, eta)
    s = solver_like(o)
    rg = s.mag_rhs(rho, e, u, Bx, By, Bz, eta)
    for key in ("de", "du", "dBx", "dBy", "dBz"):
        scale = max(np.abs(ro[key]).max(), 1e-3 * np.abs(ro["du"]).max())
        assert rel(rg[key], ro[key], scale) <= 1e-12, (key, rel(rg[key], ro[key], scale))


@pytest.mark.parametrize("mesh", [(1, 1), (1, 3), (3, 1)])
@pytest.mark.parametrize("pk", [(2, 2), (3, 3)])
def test_one_element_wide_meshes_stabilised_strang_step(mesh, pk):
    wl = workloads.orszag_tang()
    o, s = stab_pair(wl, *mesh, *pk)
    dt = o.cfl_dt()
    st_o, taken_o, _ = o.strang_step(dt)
    st_g, taken_g = s.strang_step(dt)
    assert st_o in (0, 1) and st_g == st_o and taken_g == taken_o
    compare_state(o, s, 1e-12)


def test_refined_reciprocal_against_ieee_division():
    """The reciprocal the kernels use in place of division (PTX seed plus one
    cubic Newton step) is within 1 ulp of IEEE 1/x over its stated range
    [2^-1000, 2^1000] of both signs and at the limiter's floors."""
    import torch
    from paper_2609_10849_b300.mhd import rcp_check
    rng = np.random.default_rng(5)
    e = rng.uniform(-1000.0, 1000.0, 200000)
    x = np.ldexp(rng.uniform(1.0, 2.0, e.size), np.floor(e).astype(int) - 1)
    x[::2] *= -1.0
    special = [64 * EPS, 8192 * EPS, EPS, 1.0, 2.0, 3.0, 0.1, 1.0 / 3.0, 2.0 ** -1000, 2.0 ** 999 * 1.999,
               25 / (36 * math.pi), 5 / (12 * math.pi)]
    x = np.concatenate([x, special, [-v for v in special]])
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    rcp_check(xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    want = 1.0 / x
    ulp = np.spacing(np.abs(want))
    err = np.abs(y - want) / ulp
    assert err.max() <= 1.0, (err.max(), x[err.argmax()])


def test_fast_sqrt_against_ieee_sqrt():
    """The square root the kernels use (Heron's iteration from the PTX
    rsqrt seed) is within 1 ulp of IEEE sqrt over the whole normal range,
    exact on perfect squares of small integers and powers of 4, and follows
    IEEE sqrt on zeros, subnormals, infinity, NaN and negative inputs."""
    import torch
    from paper_2609_10849_b300.mhd import sqrt_check
    rng = np.random.default_rng(11)
    e = rng.uniform(-1022.0, 1024.0, 400000)
    x = np.ldexp(rng.uniform(1.0, 2.0, e.size), np.floor(e).astype(int) - 1)
    x = x[np.isfinite(x)]
    special = [64 * EPS, 8192 * EPS, EPS, 1.0, 2.0, 3.0, 0.1, 1.0 / 3.0, 1.4 * 0.4 / 1.0, 2.0 ** -1022,
               np.nextafter(2.0 ** -1022, 1.0), np.finfo(float).max, 2.0 ** 1022 * 1.5]
    squares = [float(i * i) for i in range(1, 2000)] + [4.0 ** i for i in range(-500, 500)]
    x = np.concatenate([x, special, squares])
    edge = np.array([0.0, -0.0, 5e-324, 2.0 ** -1030, np.inf, np.nan, -1.0, -2.0 ** -1000, -np.inf])
    xd = torch.tensor(np.concatenate([x, edge]), dtype=torch.float64, device="cuda")
    yd = torch.empty_like(xd)
    sqrt_check(xd, yd)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    want = np.sqrt(x)
    err = np.abs(y[:x.size] - want) / np.spacing(want)
    assert err.max() <= 1.0, (err.max(), x[err.argmax()])
    nsq = len(squares)
    assert np.array_equal(y[x.size - nsq:x.size], want[x.size - nsq:])
    ye = y[x.size:]
    with np.errstate(invalid="ignore"):
        we = np.sqrt(edge)
    assert np.array_equal(np.isnan(ye), np.isnan(we))
    ok = ~np.isnan(we)
    assert np.array_equal(ye[ok], we[ok])
    assert np.array_equal(np.signbit(ye[ok]), np.signbit(we[ok]))
