"""The oracle's OpenMP timing build (used only to time the CPU baseline on all
cores) computes exactly what the plain build computes: its parallel element
loops write disjoint data and every sum keeps its serial order, so a
stabilised Strang step, a magnetic residual and the diagnostics agree bit for
bit with the plain build at several thread counts."""
import numpy as np
import pytest

from oracle import Oracle, ParallelOracle
from paper_2609_10849_b300 import workloads

STAB = dict(oe_hydro=1, oe_vel=1, pp=1, ar=1, s_H=0.02, s_M=0.02, C_s=5.0, C_eta=0.2)


def _start(cls, wl, nx, ny, p, k):
    o = cls(nx, ny, p, k, wl["gamma"], wl["domain"])
    X, Y = o.coords("dg")
    rho, ux, uy, uz, pr, _ = wl["fields"](X, Y)
    XW, YW = o.coords("w")
    XZ, YZ = o.coords("bz")
    Bx, By = o.b_from_potential(wl["Az"](XW, YW), *wl["B0"])
    o.set_primitive(rho, np.stack([ux, uy, uz]), pr, Bx, By, wl["fields"](XZ, YZ)[5])
    o.set_params(cfl=0.4, **STAB)
    return o


@pytest.mark.parametrize("wl_name,pk", [("orszag_tang", (3, 3)), ("blast", (2, 2)), ("orszag_tang", (3, 2))])
@pytest.mark.parametrize("threads", [3, 8])
def test_parallel_build_is_bitwise_serial(wl_name, pk, threads):
    wl = workloads.WORKLOADS[wl_name]()
    a = _start(Oracle, wl, 11, 9, *pk)
    b = _start(ParallelOracle, wl, 11, 9, *pk)
    assert b.set_threads(threads) == threads
    dt = a.cfl_dt()
    assert b.cfl_dt() == dt
    for _ in range(2):
        assert a.strang_step(dt) == b.strang_step(dt)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert np.array_equal(a.eta(), b.eta())
    da, db = a.diagnostics(), b.diagnostics()
    assert all(da[k] == db[k] for k in da)
