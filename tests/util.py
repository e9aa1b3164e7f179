"""Helpers shared by the tests: oracle states built from the workload module."""
import numpy as np

from oracle import Oracle
from paper_2609_10849_b300 import workloads


def oracle_state(wl, nx, ny, p, m, t=0.0):
    """Oracle with the nodal initial state of workload dict ``wl`` (reading R10)."""
    o = Oracle(nx, ny, p, m, wl["gamma"], wl["domain"])
    X, Y = o.coords("dg")
    kw = {"t": t} if t else {}
    rho, ux, uy, uz, pr, _ = wl["fields"](X, Y, **kw)
    XW, YW = o.coords("w")
    Bx, By = o.b_from_potential(wl["Az"](XW, YW, **kw), *wl["B0"])
    XZ, YZ = o.coords("bz")
    Bz = wl["fields"](XZ, YZ, **kw)[5]
    o.set_primitive(rho, np.stack([ux, uy, uz]), pr, Bx, By, Bz)
    return o


def prim_from_cons(U, gamma):
    rho = U[0]
    u = U[1:4] / rho
    e = (U[4] - 0.5 * rho * (u ** 2).sum(axis=0)) / rho
    return rho, u, e


def mirror_images(U, Bx, By, Bz, pnx, pny, p, m, walls, cond):
    """Reflecting walls by the method of images, written with numpy on the host
    layouts (independent of the library's kernel): the doubled periodic state
    whose physical part (ex < pnx, ey < pny) is taken from the input and whose
    image part is the mirror of it.  Normal velocity odd; B per wall pair with
    the parity of a conducting wall (cond bit set: B_n odd, B_t even; the
    normal B on the wall is zeroed) or of a symmetry plane (B_n even, B_t odd).
    Returns new arrays."""
    n, mm = p + 1, m + 1
    nx = pnx * (2 if walls & 1 else 1)
    ny = pny * (2 if walls & 2 else 1)
    U = np.array(U, dtype=np.float64).reshape(5, ny, nx, n, n).copy()
    Bx = np.array(Bx, dtype=np.float64).reshape(ny * mm, nx * mm).copy()
    By = np.array(By, dtype=np.float64).reshape(ny * mm, nx * mm).copy()
    Bz = np.array(Bz, dtype=np.float64).reshape(ny, nx, mm, mm).copy()
    NY, NX, PY, PX = ny * mm, nx * mm, pny * mm, pnx * mm
    if walls & 1:
        cx = bool(cond & 1)
        U[:, :, pnx:] = U[:, :, pnx - 1::-1, :, ::-1]
        U[1, :, pnx:] *= -1.0
        if cx:
            Bx[:, 0] = 0.0
            Bx[:, PX] = 0.0
        for c in range(PX + 1, NX):
            Bx[:, c] = (-1.0 if cx else 1.0) * Bx[:, NX - c]
        for c in range(PX, NX):
            By[:, c] = (1.0 if cx else -1.0) * By[:, NX - 1 - c]
        Bz[:, pnx:] = (1.0 if cx else -1.0) * Bz[:, pnx - 1::-1, :, ::-1]
    if walls & 2:
        cy = bool(cond & 2)
        U[:, pny:] = U[:, pny - 1::-1, :, ::-1, :]
        U[2, pny:] *= -1.0
        for r in range(PY, NY):
            Bx[r, :] = (1.0 if cy else -1.0) * Bx[NY - 1 - r, :]
        if cy:
            By[0, :] = 0.0
            By[PY, :] = 0.0
        for r in range(PY + 1, NY):
            By[r, :] = (-1.0 if cy else 1.0) * By[NY - r, :]
        Bz[pny:] = (1.0 if cy else -1.0) * Bz[pny - 1::-1, :, ::-1, :]
    return U.reshape(5, -1), Bx.ravel(), By.ravel(), Bz.ravel()


def physical_part(U, Bx, By, Bz, nx, ny, pnx, pny, p, m):
    """The physical elements' DG nodes and B_z (ex < pnx, ey < pny) of a doubled
    state, and its in-plane B on the physical rows and columns."""
    n, mm = p + 1, m + 1
    U5 = np.asarray(U).reshape(5, ny, nx, n, n)[:, :pny, :pnx]
    Bz4 = np.asarray(Bz).reshape(ny, nx, mm, mm)[:pny, :pnx]
    Bx2 = np.asarray(Bx).reshape(ny * mm, nx * mm)[:pny * mm, :pnx * mm + 1]
    By2 = np.asarray(By).reshape(ny * mm, nx * mm)[:pny * mm + 1, :pnx * mm]
    return U5, Bx2, By2, Bz4
