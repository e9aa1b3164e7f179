"""Error behaviour of the C ABI as the header states it: invalid arguments are
refused with MHD_EINVAL and a message (mhd_last_error), nothing is changed,
and a context stays usable after a refused call.

The creation checks run on the CPU: mhd_create and mhd_batch_create validate
their arguments before any CUDA call.  The rest need a context (a GPU).
"""
import numpy as np
import pytest

from paper_2609_10849_b300 import workloads
from paper_2609_10849_b300.mhd import MhdError, Solver

MHD_EINVAL = -1


@pytest.mark.parametrize("args,msg", [
    ((0, 4, 2, 2, 5 / 3), "invalid mesh"),
    ((4, 0, 2, 2, 5 / 3), "invalid mesh"),
    ((4, 4, 0, 0, 5 / 3), "unsupported"),
    ((4, 4, 5, 5, 5 / 3), "unsupported"),
    ((4, 4, 3, 1, 5 / 3), "unsupported"),
    ((4, 4, 2, 3, 5 / 3), "unsupported"),
    ((4, 4, 2, 2, 1.0), "gamma"),
    ((4, 4, 2, 2, float("nan")), "gamma"),
    ((40000, 40000, 1, 1, 5 / 3), "too large"),
])
def test_create_rejects(args, msg):
    with pytest.raises(MhdError, match=msg) as e:
        Solver(*args)
    assert e.value.code == MHD_EINVAL


@pytest.mark.parametrize("domain", [(1.0, 1.0, 0.0, 1.0), (0.0, 1.0, 0.5, -0.5)])
def test_create_rejects_empty_domain(domain):
    with pytest.raises(MhdError, match="invalid mesh"):
        Solver(4, 4, 2, 2, 5 / 3, domain)


@pytest.mark.parametrize("walls,cond", [(0, 0), (4, 0), (1, 2), (2, 1), (-1, 0), (3, 4)])
def test_create_walled_rejects(walls, cond):
    """mhd_create_walled validates its wall flags before any CUDA call."""
    with pytest.raises(MhdError, match="walls") as e:
        Solver(4, 4, 2, 2, 5 / 3, walls=walls, conducting=cond) if walls else _walled_zero()
    assert e.value.code == MHD_EINVAL


def _walled_zero():
    import ctypes as C
    from paper_2609_10849_b300 import mhd
    h = C.c_void_p()
    mesh = mhd.Mesh(4, 4, 0.0, 1.0, 0.0, 1.0)
    mhd._check(mhd.lib().mhd_create_walled(C.byref(mesh), 2, 2, 5 / 3, 0, 0, C.byref(h)))


def test_batch_create_rejects_no_runs():
    from paper_2609_10849_b300.mhd import Batch
    with pytest.raises(MhdError, match="invalid argument"):
        Batch([])


def test_static_residual_wrapper_refuses_bad_buffers_before_the_library(monkeypatch):
    """The allocation-free residual's C entry point sees bare device pointers
    and cannot check their extent, device or overlap; the binding refuses a
    tensor of the wrong size, an output that overlaps the input and tensors
    that are not on the current CUDA device before anything reaches the
    library (CPU: the library must not be touched at all)."""
    import torch
    from paper_2609_10849_b300 import mhd

    def no_library():
        raise AssertionError("the library was called")

    monkeypatch.setattr(mhd, "lib", no_library)
    nx, ny, p = 3, 2, 2
    need = 5 * nx * ny * (p + 1) ** 2
    dom = (0.0, 1.0, 0.0, 1.0)
    good = torch.zeros(need, dtype=torch.float64)
    with pytest.raises(ValueError, match="entries"):
        mhd.hydro_rhs_static(nx, ny, p, 1.4, dom, torch.zeros(need - 1, dtype=torch.float64), good)
    with pytest.raises(ValueError, match="entries"):
        mhd.hydro_rhs_static(nx, ny, p, 1.4, dom, good, torch.zeros(need + 5, dtype=torch.float64))
    with pytest.raises(ValueError, match="float64"):
        mhd.hydro_rhs_static(nx, ny, p, 1.4, dom, good.float(), good.clone())
    with pytest.raises(ValueError, match="overlap"):
        mhd.hydro_rhs_static(nx, ny, p, 1.4, dom, good, good)
    big = torch.zeros(2 * need, dtype=torch.float64)
    with pytest.raises(ValueError, match="overlap"):
        mhd.hydro_rhs_static(nx, ny, p, 1.4, dom, big[:need], big[need // 2:need // 2 + need])
    with pytest.raises(ValueError, match="CUDA"):
        mhd.hydro_rhs_static(nx, ny, p, 1.4, dom, good, good.clone())
    with pytest.raises(ValueError, match="torch tensor"):
        mhd.hydro_rhs_static(nx, ny, p, 1.4, dom, np.zeros(need), good)


def _small():
    wl = workloads.orszag_tang()
    s = Solver(4, 3, 2, 2, wl["gamma"], wl["domain"])
    X, Y = s.coords("dg")
    rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
    s.set_primitive(rho, np.stack([ux, uy, uz]), pr)
    XW, YW = s.coords("w")
    XZ, YZ = s.coords("bz")
    s.set_B_from_potential(wl["Az"](XW, YW), *wl["B0"], wl["fields"](XZ, YZ)[5])
    return s


@pytest.mark.gpu
def test_refused_calls_leave_the_context_usable():
    s = _small()
    ref = _small()
    before = [a.copy() for a in s.get_state()]
    for kw in (dict(cfl=0.0), dict(s_H=-1.0), dict(C_eta=-0.1), dict(max_halvings=-1), dict(strang_order=2)):
        with pytest.raises(MhdError, match="invalid stabilisation parameters"):
            s.set_params(**kw)
    assert s.params == ref.params  # the refused values were not kept
    with pytest.raises(MhdError, match="invalid argument"):
        s.substep("M", 0.0)
    with pytest.raises(MhdError, match="invalid argument"):
        s.strang_steps(-1e-3, 2)
    with pytest.raises(MhdError, match="invalid argument"):
        s.strang_steps(1e-3, -1)
    assert s.strang_steps(1e-3, 0) == 0
    with pytest.raises(MhdError, match="invalid tile variant"):
        s.set_tiles(9, 0)
    with pytest.raises(MhdError, match="invalid tile variant"):
        s.set_tiles(0, 27)
    with pytest.raises(MhdError, match="invalid tile variant"):
        s.set_tiles(0, -1)
    with pytest.raises(MhdError, match="nq"):
        s.quad_coords(0)
    with pytest.raises(MhdError, match="nq"):
        s.quad_coords(17)
    X, Y = s.quad_coords(2)
    with pytest.raises(MhdError, match="nq"):
        s.set_Bz_projected(np.zeros_like(X), 2)  # k = 2 needs nq >= 3
    x = np.zeros(s.state_size())
    with pytest.raises(MhdError, match="invalid argument"):
        s.adjoint_segment(x, 0, x, 1e-3)
    for a, b in zip(s.get_state(), before):
        assert np.array_equal(a, b)
    # the context still steps exactly like a fresh one
    assert s.strang_steps(1e-3, 3) == 3
    assert ref.strang_steps(1e-3, 3) == 3
    for a, b in zip(s.get_state(), ref.get_state()):
        assert np.array_equal(a, b)


@pytest.mark.gpu
def test_adjoint_refuses_mhm_order():
    s = _small()
    s.set_params(strang_order=1)
    with pytest.raises(MhdError):
        s.adjoint_segment(np.ones(s.state_size()), 1, np.ones(s.state_size()), 1e-3)


@pytest.mark.gpu
def test_host_and_device_buffers_do_not_mix():
    import torch
    s = _small()
    U, Bx, By, Bz = s.get_state()
    with pytest.raises(ValueError, match="mix of host and device"):
        s.set_state(torch.tensor(U, device="cuda"), Bx, By, Bz)
    with pytest.raises(ValueError, match="float64"):
        s.set_state(U.astype(np.float32), Bx, By, Bz)


@pytest.mark.gpu
def test_reduced_2d2v_refuses_out_of_plane_fields():
    """The reduced 2D2V stage is exact only for u_z = B_z = 0: on a state with
    B_z != 0 every stepping call refuses it, leaves the state as it was, and
    the same context steps normally once the full stage is selected again."""
    from tests.util import oracle_state
    wl = workloads.alfven_diagonal()  # B_z and u_z nonzero
    o = oracle_state(wl, 4, 4, 2, 2)
    s = Solver(4, 4, 2, 2, wl["gamma"], wl["domain"])
    s.set_state(*o.get_state())
    s.set_params(reduced_2d2v=1)
    before = [a.copy() for a in s.get_state()]
    with pytest.raises(MhdError, match="reduced_2d2v needs") as e:
        s.strang_step(1e-3)
    assert e.value.code == MHD_EINVAL
    with pytest.raises(MhdError, match="reduced_2d2v needs"):
        s.strang_steps(1e-3, 2)
    with pytest.raises(MhdError, match="reduced_2d2v needs"):
        s.substep("M", 1e-3)
    for a, b in zip(s.get_state(), before):
        assert np.array_equal(a, b)
    s.set_params(reduced_2d2v=0)
    assert s.strang_steps(1e-3, 2) == 2
