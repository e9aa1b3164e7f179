"""Adjoint of the CUDA path (hand-written vector-Jacobian products through the
C ABI) against the oracle's forward-mode tangent and against central finite
differences of the CUDA forward.

* residual VJPs: the full Jacobian on tiny meshes element by element
  (rows from the GPU VJP with unit adjoints, columns from the oracle tangent
  with unit directions), and the dot-product test <lam, J dx> = <J^T lam, dx>
  on larger meshes for every (p, k);
* one Strang step: the dot-product test against the oracle tangent of the
  whole step;
* a differentiable sequence of steps with checkpointing (torch.autograd):
  directional derivatives of an objective against central differences.

Tolerances: Jacobian entries 1e-11 of the largest entry; dot products 1e-12 of
sum |lam_i (J dx)_i| (both sides are exact up to rounding); finite differences
1e-6 relative (the accuracy bar of the adjoint).
"""
import numpy as np
import pytest

from oracle import Oracle, Tangent
from tests.test_oracle_magnetic import random_mag_state
from tests.test_oracle_tangent import generic_state

pytestmark = pytest.mark.gpu

PK = [(1, 0), (1, 1), (2, 1), (2, 2), (3, 2), (3, 3), (4, 3), (4, 4)]


def solver_like(o):
    from paper_2609_10849_b300.mhd import Solver
    return Solver(o.nx, o.ny, o.p, o.m, o.gamma, o.domain)


def dot_check(lam, Jdx, JTlam, dx, tol=1e-12):
    a = sum(float((l * j).sum()) for l, j in zip(lam, Jdx))
    b = sum(float((g * d).sum()) for g, d in zip(JTlam, dx))
    scale = sum(float(np.abs(l * j).sum()) for l, j in zip(lam, Jdx))
    assert abs(a - b) <= tol * scale, (a, b, abs(a - b) / scale)


@pytest.mark.parametrize("p", [1, 2])
def test_hydro_vjp_full_jacobian(p):
    rng = np.random.default_rng(800 + p)
    dom = (0.0, 1.0, 0.0, 0.8)
    t = Tangent(2, 2, p, p, 1.4, dom)
    U = generic_state(t, rng)
    n = U.size
    Jt = np.zeros((n, n))  # columns from the tangent
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        Jt[:, j] = t.hydro_rhs_tangent(U, e.reshape(U.shape))[1].ravel()
    s = solver_like(t)
    Jg = np.zeros((n, n))  # rows from the VJP
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        Jg[i, :] = s.hydro_rhs_vjp(U, e.reshape(U.shape)).ravel()
    assert np.abs(Jg - Jt).max() <= 1e-11 * np.abs(Jt).max()


@pytest.mark.parametrize("p", [1, 2])
def test_hydro_vjp_full_jacobian_strong_variation(p):
    """Nodal densities and pressures varying by factors of order e inside an
    element: many pairs take the logarithm branch of the log mean (and its
    derivative), and the volume kernel's per-node logarithms are formed."""
    rng = np.random.default_rng(820 + p)
    dom = (0.0, 1.0, 0.0, 0.8)
    t = Tangent(2, 2, p, p, 1.4, dom)
    shape = generic_state(t, rng).shape
    rho = np.exp(0.4 * rng.standard_normal(shape[1:]))
    pr = np.exp(0.4 * rng.standard_normal(shape[1:]))
    u = np.stack([0.4 + 0.1 * rng.standard_normal(shape[1:]), 0.3 + 0.1 * rng.standard_normal(shape[1:]),
                  0.1 * rng.standard_normal(shape[1:])])
    U = np.concatenate([rho[None], rho * u, (pr / 0.4 + 0.5 * rho * (u * u).sum(0))[None]])
    n = U.size
    Jt = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        Jt[:, j] = t.hydro_rhs_tangent(U, e.reshape(U.shape))[1].ravel()
    s = solver_like(t)
    Jg = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        Jg[i, :] = s.hydro_rhs_vjp(U, e.reshape(U.shape)).ravel()
    assert np.abs(Jg - Jt).max() <= 1e-11 * np.abs(Jt).max()


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("mesh", [(5, 4), (3, 7)])
def test_hydro_vjp_dot(p, mesh):
    rng = np.random.default_rng(810 + 10 * p + mesh[0])
    t = Tangent(*mesh, p, p, 1.4, (0.0, 1.0, 0.0, 0.8))
    U = generic_state(t, rng)
    dU = rng.standard_normal(U.shape)
    lam = rng.standard_normal(U.shape)
    dL = t.hydro_rhs_tangent(U, dU)[1]
    g = solver_like(t).hydro_rhs_vjp(U, lam)
    dot_check([lam], [dL], [g], [dU])


def mag_inputs(o, rng):
    rho, e, u, Bx, By, Bz = random_mag_state(o, rng)
    return dict(rho=rho, e=e, u=u, Bx=Bx, By=By, Bz=Bz)


@pytest.mark.parametrize("pk", [(1, 0), (1, 1), (2, 1)])
def test_mag_vjp_full_jacobian(pk):
    p, k = pk
    rng = np.random.default_rng(830 + 10 * p + k)
    t = Tangent(2, 2, p, k, 5 / 3, (0.0, 1.3, 0.0, 0.7))
    st = mag_inputs(t, rng)
    keys_in = ("rho", "u", "Bx", "By", "Bz")
    sizes_in = [np.size(st[k_]) for k_ in keys_in]
    keys_out = ("du", "dBx", "dBy", "dBz")
    zero = {k_: np.zeros(np.shape(v)) for k_, v in st.items()}
    n_in = sum(sizes_in)
    cols = []
    for j in range(n_in):
        tang = {k_: v.copy() for k_, v in zero.items()}
        off = j
        for k_, sz in zip(keys_in, sizes_in):
            if off < sz:
                tang[k_].reshape(-1)[off] = 1.0
                break
            off -= sz
        r, dr = t.mag_rhs_tangent(st, tang)
        cols.append(np.concatenate([np.ravel(dr[k_]) for k_ in keys_out]))
    Jt = np.stack(cols, axis=1)
    s = solver_like(t)
    n_out = Jt.shape[0]
    N = t.K * t.n2
    Jg = np.zeros_like(Jt)
    for i in range(n_out):
        w = np.zeros(n_out)
        w[i] = 1.0
        wu, wBx, wBy, wBz = np.split(w, np.cumsum([3 * N, t.G, t.G]))
        g = s.mag_rhs_vjp(st["rho"], st["u"], st["Bx"], st["By"], st["Bz"], wu.reshape(3, N), wBx, wBy, wBz)
        Jg[i, :] = np.concatenate([np.ravel(a) for a in g])
    assert np.abs(Jg - Jt).max() <= 1e-11 * np.abs(Jt).max()


@pytest.mark.parametrize("pk", PK)
def test_mag_vjp_dot(pk):
    p, k = pk
    rng = np.random.default_rng(850 + 10 * p + k)
    t = Tangent(5, 3, p, k, 5 / 3, (0.0, 1.3, 0.0, 0.7))
    st = mag_inputs(t, rng)
    tang = {k_: rng.standard_normal(np.shape(v)) for k_, v in st.items()}
    tang["e"][:] = 0.0  # the ideal residual does not depend on e
    _, dr = t.mag_rhs_tangent(st, tang)
    w = {k_: rng.standard_normal(np.shape(dr[k_])) for k_ in ("du", "dBx", "dBy", "dBz")}
    s = solver_like(t)
    g = s.mag_rhs_vjp(st["rho"], st["u"], st["Bx"], st["By"], st["Bz"], w["du"], w["dBx"], w["dBy"], w["dBz"])
    dot_check([w["du"], w["dBx"], w["dBy"], w["dBz"]], [dr["du"], dr["dBx"], dr["dBy"], dr["dBz"]], g,
              [tang["rho"], tang["u"], tang["Bx"], tang["By"], tang["Bz"]])
    assert np.abs(dr["de"]).max() == 0.0


def packed(o, U, Bx, By, Bz):
    return np.concatenate([np.ravel(U), Bx, By, Bz])


@pytest.mark.parametrize("pk", [(1, 1), (2, 2), (3, 2), (3, 3), (4, 4)])
def test_adjoint_step_dot(pk):
    p, k = pk
    rng = np.random.default_rng(870 + 10 * p + k)
    dom = (0.0, 1.0, 0.0, 1.0)
    t = Tangent(4, 3, p, k, 5 / 3, dom)
    U = generic_state(t, rng)
    Bx, By = rng.uniform(-0.5, 0.5, t.G), rng.uniform(-0.5, 0.5, t.G)
    Bz = rng.uniform(-0.5, 0.5, t.Z)
    x = [U, Bx, By, Bz]
    dx = [rng.standard_normal(np.shape(a)) for a in x]
    dt = 1e-3
    t.set_state(*x)
    t.set_tangent(*dx)
    assert t.strang_step(dt)[0] == 0
    Jdx = t.get_tangent()
    s = solver_like(t)
    lam = [rng.standard_normal(np.shape(a)) for a in x]
    g = s.adjoint_step(packed(t, *x), packed(t, *lam), dt)
    gs = np.split(g, np.cumsum([U.size, t.G, t.G]))
    dot_check([np.ravel(a) for a in lam], [np.ravel(a) for a in Jdx], gs, [np.ravel(a) for a in dx])


def test_adjoint_reports_frozen_maps():
    rng = np.random.default_rng(890)
    t = Tangent(3, 3, 2, 2, 5 / 3)
    U = generic_state(t, rng)
    s = solver_like(t)
    x = packed(t, U, np.zeros(t.G), np.zeros(t.G), np.zeros(t.Z))
    s.adjoint_step(x, x.copy(), 1e-3)
    assert s.last_adjoint_flags == 0
    s.set_params(oe_hydro=1, pp=1, ar=1, C_eta=0.2, oe_vel=1)
    s.adjoint_step(x, x.copy(), 1e-3)
    assert s.last_adjoint_flags == 1 | 2 | 4 | 8


@pytest.mark.parametrize("pk,oe", [((2, 2), 1), ((3, 3), 1), ((4, 3), 1), ((2, 2), 0), ((4, 3), 0)])
def test_adjoint_step_frozen_stage_maps_dot(pk, oe):
    """Hydro OE (oe = 1) and limiter on: the adjoint with frozen D_l and theta
    against the oracle tangent with the same coefficients held at their values.
    A few nodes of the state are near vacuum in pressure; with the OE off the
    limiter acts on them (without it the step would be rejected)."""
    p, k = pk
    rng = np.random.default_rng(900 + 10 * p + k)
    dom = (0.0, 1.0, 0.0, 1.0)
    t = Tangent(5, 4, p, k, 5 / 3, dom)
    prm = dict(oe_hydro=oe, pp=1, s_H=0.5)
    t.set_params(**prm)
    t.set_frozen(True)
    U = generic_state(t, rng)
    for q in (7, 40, 63):  # E = kinetic energy + a tiny internal energy
        kin = 0.5 * (U[1, q] ** 2 + U[2, q] ** 2 + U[3, q] ** 2) / U[0, q]
        U[4, q] = kin + 1e-9
    Bx, By = rng.uniform(-0.5, 0.5, t.G), rng.uniform(-0.5, 0.5, t.G)
    Bz = rng.uniform(-0.5, 0.5, t.Z)
    x = [U, Bx, By, Bz]
    dx = [rng.standard_normal(np.shape(a)) for a in x]
    dt = 2e-3
    t.set_state(*x)
    t.set_tangent(*dx)
    assert t.strang_step(dt)[0] == 0
    Jdx = t.get_tangent()
    s = solver_like(t)
    s.set_params(**prm)
    lam = [rng.standard_normal(np.shape(a)) for a in x]
    g = s.adjoint_step(packed(t, *x), packed(t, *lam), dt)
    gs = np.split(g, np.cumsum([U.size, t.G, t.G]))
    # the frozen coefficients of the two sides agree to rounding, amplified
    # through the sensor's quotients
    dot_check([np.ravel(a) for a in lam], [np.ravel(a) for a in Jdx], gs, [np.ravel(a) for a in dx], tol=1e-9)


def vortex_problem(n, p, dt_steps_cfl=True):
    """Advected MHD vortex (§4.2) on an n x n mesh: solver, packed magnetic part,
    nodal rho0, u0, p0 and the CFL step at t = 0."""
    import torch
    from paper_2609_10849_b300 import workloads
    from paper_2609_10849_b300.mhd import Solver
    wl = workloads.balsara_vortex()
    s = Solver(n, n, p, p, wl["gamma"], wl["domain"])
    X, Y = s.coords("dg")
    rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
    XW, YW = s.coords("w")
    XZ, YZ = s.coords("bz")
    s.set_primitive(rho, np.stack([ux, uy, uz]), pr)
    s.set_B_from_potential(wl["Az"](XW, YW), *wl["B0"], wl["fields"](XZ, YZ)[5])
    dt = s.compute_dt()
    x = torch.zeros(s.state_size(), dtype=torch.float64, device="cuda")
    s.get_packed(x)
    B = x[5 * s.N:].clone()
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    return s, B, t(rho), t(np.stack([ux, uy, uz])), t(pr), dt, (X, Y)


def objective_setup(n, p, nsteps, every):
    import torch
    from paper_2609_10849_b300.adjoint import pack_primitive, strang_steps
    s, B, rho0, u0, p0, dt, (X, Y) = vortex_problem(n, p)
    g = s.gamma
    # target: the end state of the run started from the perturbed density
    from paper_2609_10849_b300.workloads import vortex_target_density
    rs = torch.tensor(vortex_target_density(X, Y), dtype=torch.float64, device="cuda")
    with torch.no_grad():
        xt = strang_steps(s, pack_primitive(s, rs, u0, p0, B), dt, nsteps, every)
    rho_t = xt[:s.N].clone()
    from oracle import rule
    _, w = rule("gll", p)
    hx = 10.0 / n
    Mq = torch.tensor(np.tile(np.outer(w, w).ravel() * hx * hx / 4, s.K), device="cuda")

    def J(rho, u):
        x = strang_steps(s, pack_primitive(s, rho, u, p0, B), dt, nsteps, every)
        return 0.5 * (Mq * (x[:s.N] - rho_t) ** 2).sum()

    return J, rho0, u0


@pytest.mark.parametrize("nsteps,every", [(6, 4), (5, 5)])
def test_autograd_gradient_fd(nsteps, every):
    import torch
    J, rho0, u0 = objective_setup(8, 3, nsteps, every)
    rho = rho0.clone().requires_grad_(True)
    u = u0.clone().requires_grad_(True)
    val = J(rho, u)
    val.backward()
    gen = torch.Generator(device="cuda").manual_seed(5)
    for _ in range(2):
        dr = torch.randn(rho.shape, generator=gen, device="cuda", dtype=torch.float64)
        du = torch.randn(u.shape, generator=gen, device="cuda", dtype=torch.float64)
        eps = 1e-5
        with torch.no_grad():
            jp = J(rho0 + eps * dr, u0 + eps * du).item()
            jm = J(rho0 - eps * dr, u0 - eps * du).item()
        fd = (jp - jm) / (2 * eps)
        ad = float((rho.grad * dr).sum() + (u.grad * du).sum())
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


def test_vortex_adjoint_full_size():
    """The adjoint workload at full size: 128 x 128 elements, p = k = 4, 200
    Strang steps at the t = 0 CFL step, checkpoints every 20; the gradient with
    respect to the initial density and velocity against central differences."""
    import torch
    J, rho0, u0 = objective_setup(128, 4, 200, 20)
    rho = rho0.clone().requires_grad_(True)
    u = u0.clone().requires_grad_(True)
    J(rho, u).backward()
    gen = torch.Generator(device="cuda").manual_seed(11)
    dr = torch.randn(rho.shape, generator=gen, device="cuda", dtype=torch.float64)
    du = torch.randn(u.shape, generator=gen, device="cuda", dtype=torch.float64)
    eps = 1e-5
    with torch.no_grad():
        fd = (J(rho0 + eps * dr, u0 + eps * du).item() - J(rho0 - eps * dr, u0 - eps * du).item()) / (2 * eps)
    ad = float((rho.grad * dr).sum() + (u.grad * du).sum())
    assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)


@pytest.mark.parametrize("pk", [(1, 1), (2, 2), (3, 3), (4, 4)])
def test_adjoint_step_frozen_velocity_oe_dot(pk):
    """Velocity OE on (and hydro OE, limiter): the adjoint with frozen D_l and
    rho-weighted projector against the oracle tangent holding the same
    coefficients at their values."""
    p, k = pk
    rng = np.random.default_rng(950 + 10 * p + k)
    dom = (0.0, 1.0, 0.0, 1.0)
    t = Tangent(4, 5, p, k, 5 / 3, dom)
    prm = dict(oe_hydro=1, pp=1, oe_vel=1, s_H=0.2, s_M=0.5)
    t.set_params(**prm)
    t.set_frozen(True)
    U = generic_state(t, rng)
    Bx, By = rng.uniform(-0.5, 0.5, t.G), rng.uniform(-0.5, 0.5, t.G)
    Bz = rng.uniform(-0.5, 0.5, t.Z)
    x = [U, Bx, By, Bz]
    dx = [rng.standard_normal(np.shape(a)) for a in x]
    dt = 2e-3
    t.set_state(*x)
    t.set_tangent(*dx)
    assert t.strang_step(dt)[0] == 0
    Jdx = t.get_tangent()
    s = solver_like(t)
    s.set_params(**prm)
    lam = [rng.standard_normal(np.shape(a)) for a in x]
    g = s.adjoint_step(packed(t, *x), packed(t, *lam), dt)
    gs = np.split(g, np.cumsum([U.size, t.G, t.G]))
    dot_check([np.ravel(a) for a in lam], [np.ravel(a) for a in Jdx], gs, [np.ravel(a) for a in dx], tol=1e-9)


@pytest.mark.parametrize("pk", [(1, 0), (2, 1), (3, 3), (4, 4)])
def test_adjoint_step_frozen_resistivity_dot(pk):
    """Every stabilisation map on, A.R. included: the adjoint with eta frozen
    (resistive Ohm load and Ohmic heating differentiated) against the oracle
    tangent holding the same coefficients at their values."""
    p, k = pk
    rng = np.random.default_rng(970 + 10 * p + k)
    dom = (0.0, 1.0, 0.0, 1.0)
    t = Tangent(4, 5, p, k, 5 / 3, dom)
    prm = dict(oe_hydro=1, pp=1, oe_vel=1, ar=1, C_eta=0.2, s_H=0.2, s_M=0.5)
    t.set_params(**prm)
    t.set_frozen(True)
    U = generic_state(t, rng)
    Bx, By = rng.uniform(-0.5, 0.5, t.G), rng.uniform(-0.5, 0.5, t.G)
    Bz = rng.uniform(-0.5, 0.5, t.Z)
    x = [U, Bx, By, Bz]
    dx = [rng.standard_normal(np.shape(a)) for a in x]
    dt = 2e-3
    t.set_state(*x)
    t.set_tangent(*dx)
    assert t.strang_step(dt)[0] == 0
    assert t.eta().max() > 0
    Jdx = t.get_tangent()
    s = solver_like(t)
    s.set_params(**prm)
    lam = [rng.standard_normal(np.shape(a)) for a in x]
    g = s.adjoint_step(packed(t, *x), packed(t, *lam), dt)
    gs = np.split(g, np.cumsum([U.size, t.G, t.G]))
    dot_check([np.ravel(a) for a in lam], [np.ravel(a) for a in Jdx], gs, [np.ravel(a) for a in dx], tol=1e-9)


def test_adjoint_segment_matches_steps():
    """The segment adjoint (one recorded forward pass) equals the chain of
    single-step adjoints on recomputed states, bit for bit."""
    rng = np.random.default_rng(990)
    p = k = 3
    t = Tangent(5, 4, p, k, 5 / 3, (0.0, 1.0, 0.0, 1.0))
    U = generic_state(t, rng)
    Bx, By = rng.uniform(-0.5, 0.5, t.G), rng.uniform(-0.5, 0.5, t.G)
    Bz = rng.uniform(-0.5, 0.5, t.Z)
    s = solver_like(t)
    s.set_params(oe_hydro=1, pp=1, oe_vel=1, ar=1, C_eta=0.2)
    x0 = packed(t, U, Bx, By, Bz)
    dt = 1e-3
    states = [x0]
    s.set_packed(x0)
    for _ in range(3):
        assert s.strang_step(dt)[0] == 0
        states.append(s.get_packed(np.zeros_like(x0)))
    lam = rng.standard_normal(x0.shape)
    seg = s.adjoint_segment(x0, 4, lam, dt)
    chain = lam.copy()
    for i in reversed(range(4)):
        chain = s.adjoint_step(states[i], chain, dt)
    assert np.array_equal(seg, chain)
    assert s.last_adjoint_flags == 15


def test_adjoint_with_reduced_2d2v_stage():
    """On a 2D2V state (u_z = B_z = 0) the adjoint of a solver stepping with the
    reduced magnetic stage equals that of the full stage bit for bit (its
    recomputation runs the full stage; the reduced velocity OE keeps the same
    frozen coefficients), for every stabilisation map on."""
    rng = np.random.default_rng(995)
    p = k = 3
    t = Tangent(5, 4, p, k, 5 / 3, (0.0, 1.0, 0.0, 1.0))
    U = generic_state(t, rng)
    U[3] = 0.0  # m_z
    Bx, By = rng.uniform(-0.5, 0.5, t.G), rng.uniform(-0.5, 0.5, t.G)
    Bz = np.zeros(t.Z)
    x0 = packed(t, U, Bx, By, Bz)
    lam = rng.standard_normal(x0.shape)
    out = []
    for reduced in (0, 1):
        s = solver_like(t)
        s.set_params(oe_hydro=1, pp=1, oe_vel=1, ar=1, C_eta=0.2, reduced_2d2v=reduced)
        out.append((s.adjoint_segment(x0, 3, lam, 1e-3), s.last_adjoint_flags))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


def test_primitive_exchange_and_its_vjp():
    """The input exchange U(rho, u, p) of the differentiable path runs in the
    library: its value against the oracle's exchange, and its VJP against the
    oracle's directional derivative: U is a polynomial of degree 3 in
    (rho, u, p) (E holds rho |u|^2 / 2), so the Richardson combination
    (4 D(eps) - D(2 eps)) / 3 of two central differences of the oracle's
    exchange is exact up to rounding; <lam, J d> = <J^T lam, d> at 1e-12."""
    import torch
    from paper_2609_10849_b300.mhd import Solver
    rng = np.random.default_rng(17)
    o = Oracle(5, 4, 3, 3, 1.4)
    s = Solver(5, 4, 3, 3, 1.4)
    N = o.K * o.n2
    rho = rng.uniform(0.5, 2.0, N)
    u = rng.uniform(-1.0, 1.0, (3, N))
    p = rng.uniform(0.2, 1.5, N)
    z, zb = np.zeros(o.G), np.zeros(o.Z)

    def oracle_U(r, v, q):
        o.set_primitive(r, v, q, z, z, zb)
        return o.get_state()[0]

    U = np.zeros((5, N))
    s.primitive_to_conservative(rho, np.ascontiguousarray(u), p, U)
    Uo = oracle_U(rho, u, p)
    assert np.abs(U - Uo).max() <= 1e-14 * np.abs(Uo).max()
    dr, du, dp = rng.standard_normal(N), rng.standard_normal((3, N)), rng.standard_normal(N)
    def central(eps):
        return (oracle_U(rho + eps * dr, u + eps * du, p + eps * dp)
                - oracle_U(rho - eps * dr, u - eps * du, p - eps * dp)) / (2 * eps)

    jd = (4.0 * central(1e-2) - central(2e-2)) / 3.0
    lam = rng.standard_normal((5, N))
    t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g_rho, g_u, g_p = torch.empty(N, dtype=torch.float64, device="cuda"), t(np.zeros((3, N))), \
        torch.empty(N, dtype=torch.float64, device="cuda")
    s.primitive_to_conservative_vjp(t(rho), t(u), t(lam), g_rho, g_u, g_p)
    lhs = float((lam * jd).sum())
    rhs = float((g_rho.cpu().numpy() * dr).sum() + (g_u.cpu().numpy() * du).sum() + (g_p.cpu().numpy() * dp).sum())
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(lam).sum() * np.abs(jd).max()), (lhs, rhs)
