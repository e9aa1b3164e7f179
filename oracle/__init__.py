"""Plain FP64 CPU oracle of the H-M-H Strang step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``liboracle.so`` (built from
``mhd_oracle.cpp`` by :func:`build`) with ctypes and exchanges numpy arrays in
the host layouts of the C-ABI:

* DG nodal fields ``[K, (p+1)^2]``, ``K = ey*nx + ex``, node ``j*(p+1)+i``;
* ``Bx``, ``By``, ``Ex``/``Jx`` … on ``[ny*(m+1), nx*(m+1)]`` grids;
* ``Bz`` on ``[K, (m+1)^2]`` GLL(m) nodes.

Every function cites the section or equation of the paper it follows inside the
C++ source.  Nothing here imports the CUDA package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.cpp")
_INC = os.path.join(_HERE, "mhd_oracle_stab.inc")
_DUAL = os.path.join(_HERE, "dual.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_T = os.path.join(_HERE, "liboracle_tangent.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")

OK, RETRIED, REJECT, INADMISSIBLE = 0, 1, -10, -11


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain -O2, no FMA contraction), its forward-mode
    tangent build liboracle_tangent.so (same source, dual-number scalar) and
    the OpenMP timing build liboracle_omp.so (same source and flags plus
    -fopenmp: independent element loops on threads, every sum in its serial
    order, so its results equal the plain build's bit for bit) if they are
    stale."""
    for out, extra in ((_LIB, []), (_LIB_T, ["-DORACLE_TANGENT"]), (_LIB_OMP, ["-fopenmp"])):
        stale = force or not os.path.exists(out) or any(
            os.path.getmtime(s) > os.path.getmtime(out) for s in (_SRC, _INC, _DUAL))
        if stale:
            subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", *extra,
                                   "-shared", "-o", out + ".tmp", _SRC], cwd=_HERE)
            os.replace(out + ".tmp", out)
    return _LIB


_lib = None
_lib_t = None
_lib_omp = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def _load(path):
    L = C.CDLL(path)
    L.or_rule.argtypes = [C.c_int, C.c_int, _dp, _dp]
    L.or_lagrange.argtypes = [_dp, C.c_int, C.c_int, C.c_double, C.c_int]
    L.or_lagrange.restype = C.c_double
    L.or_log_mean.argtypes = [C.c_double, C.c_double]
    L.or_log_mean.restype = C.c_double
    for f in ("or_ec_flux", "or_llf_flux"):
        getattr(L, f).argtypes = [C.c_int, _dp, _dp, C.c_double, _dp]
    L.or_phys_flux.argtypes = [C.c_int, _dp, C.c_double, _dp]
    L.or_create.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                            C.c_int, C.c_int, C.c_double]
    L.or_create.restype = C.c_void_p
    L.or_destroy.argtypes = [C.c_void_p]
    L.or_set_params.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int]
    L.or_coords.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
    L.or_b_from_potential.argtypes = [C.c_void_p, _dp, C.c_double, C.c_double, _dp, _dp]
    L.or_set_state.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
    L.or_get_state.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
    L.or_hydro_rhs.argtypes = [C.c_void_p, _dp, _dp]
    L.or_mag_rhs.argtypes = [C.c_void_p] + [_dp] * 14
    L.or_mag_product.argtypes = [C.c_void_p] + [_dp] * 6
    L.or_mag_product.restype = C.c_double
    L.or_substep.argtypes = [C.c_void_p, C.c_int, C.c_double]
    L.or_strang_step.argtypes = [C.c_void_p, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.or_cfl_dt.argtypes = [C.c_void_p]
    L.or_cfl_dt.restype = C.c_double
    L.or_div_metric.argtypes = [C.c_void_p]
    L.or_div_metric.restype = C.c_double
    L.or_get_eta.argtypes = [C.c_void_p, _dp]
    L.or_set_eta.argtypes = [C.c_void_p, _dp]
    L.or_diagnostics.argtypes = [C.c_void_p, _dp]
    L.or_sample.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp, _dp, _dp, _dp]
    L.or_quad_coords.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
    L.or_project_Bz.argtypes = [C.c_void_p, _dp, C.c_int]
    L.or_hydro_stage_map.argtypes = [C.c_void_p, _dp, C.c_double]
    L.or_oe_sensor.argtypes = [C.c_void_p, _dp, C.c_int, _dp]
    L.or_ar_coefficient.argtypes = [C.c_void_p] + [_dp] * 6
    L.or_vel_oe.argtypes = [C.c_void_p] + [_dp] * 6 + [C.c_double]
    L.or_set_frozen.argtypes = [C.c_void_p, C.c_int]
    L.or_set_strang_order.argtypes = [C.c_void_p, C.c_int]
    L.or_threads.argtypes = [C.c_int]
    L.or_threads.restype = C.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _load(_LIB)
    return _lib


def tangent_lib():
    """The forward-mode tangent build (dual numbers; values equal the plain build's)."""
    global _lib_t
    if _lib_t is None:
        build()
        L = _load(_LIB_T)
        L.or_set_tangent.argtypes = [C.c_void_p] + [_dp] * 4
        L.or_get_tangent.argtypes = [C.c_void_p] + [_dp] * 4
        L.or_hydro_rhs_tangent.argtypes = [C.c_void_p] + [_dp] * 4
        L.or_mag_rhs_tangent.argtypes = [C.c_void_p] + [_dp] * 23
        _lib_t = L
    return _lib_t


def omp_lib():
    """The OpenMP timing build (results bitwise equal to :func:`lib`'s)."""
    global _lib_omp
    if _lib_omp is None:
        build()
        _lib_omp = _load(_LIB_OMP)
    return _lib_omp


def rule(kind: str, r: int):
    """1D rule of degree r: ``kind='gauss'`` (r+1 Gauss points) or ``'gll'``."""
    x = np.zeros(r + 2)
    w = np.zeros(r + 2)
    n = lib().or_rule(0 if kind == "gauss" else 1, r, x, w)
    return x[:n].copy(), w[:n].copy()


def lagrange(nodes, j, x, deriv=False):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    return lib().or_lagrange(nodes, len(nodes), j, float(x), int(deriv))


def log_mean(a, b):
    return lib().or_log_mean(float(a), float(b))


def _flux(fn, d, a, b, g):
    F = np.zeros(5)
    fn(d, np.ascontiguousarray(a, dtype=np.float64), np.ascontiguousarray(b, dtype=np.float64), g, F)
    return F


def ec_flux(d, UL, UR, g):
    return _flux(lib().or_ec_flux, d, UL, UR, g)


def llf_flux(d, Um, Up, g):
    return _flux(lib().or_llf_flux, d, Um, Up, g)


def phys_flux(d, U, g):
    F = np.zeros(5)
    lib().or_phys_flux(d, np.ascontiguousarray(U, dtype=np.float64), g, F)
    return F


class Oracle:
    """One mesh/discretisation of the oracle with its state."""

    def __init__(self, nx, ny, p, m, gamma, domain=(0.0, 1.0, 0.0, 1.0)):
        self.nx, self.ny, self.p, self.m, self.gamma = nx, ny, p, m, gamma
        self.domain = tuple(float(v) for v in domain)
        self.K = nx * ny
        self.n2 = (p + 1) ** 2
        self.mm = m + 1
        self.G = nx * ny * self.mm * self.mm
        self.Z = self.K * self.mm * self.mm
        self._L = self._library()
        self._h = self._L.or_create(nx, ny, *self.domain, p, m, gamma)
        if not self._h:
            raise ValueError("invalid oracle discretisation")
        self.set_params()

    @staticmethod
    def _library():
        return lib()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.or_destroy(h)
            self._h = None

    # -- configuration -----------------------------------------------------
    def set_params(self, oe_hydro=0, oe_vel=0, pp=0, ar=0, s_H=0.02, s_M=0.02, C_s=5.0, C_eta=0.0,
                   cfl=0.4, max_halvings=20, ec_faces=0):
        self._L.or_set_params(self._h, oe_hydro, oe_vel, pp, ar, s_H, s_M, C_s, C_eta, cfl,
                            max_halvings, ec_faces)

    def set_strang_order(self, order):
        """0: H-M-H (eq. strang-composition, Algorithm 3); 1: M-H-M."""
        self._L.or_set_strang_order(self._h, int(order))

    def coords(self, which):
        """Node coordinates: 'dg' [K,n2], 'w' [NY,NX], 'bz' [K,mm^2]."""
        size = {"dg": self.K * self.n2, "w": self.G, "bz": self.Z}[which]
        X = np.zeros(size)
        Y = np.zeros(size)
        self._L.or_coords(self._h, {"dg": 0, "w": 1, "bz": 2}[which], X, Y)
        return X, Y

    def b_from_potential(self, Az, Bx0=0.0, By0=0.0):
        Bx = np.zeros(self.G)
        By = np.zeros(self.G)
        self._L.or_b_from_potential(self._h, np.ascontiguousarray(Az, dtype=np.float64), Bx0, By0, Bx, By)
        return Bx, By

    # -- state -------------------------------------------------------------
    def set_state(self, U, Bx, By, Bz):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64).ravel()
        self._L.or_set_state(self._h, f(U), f(Bx), f(By), f(Bz))

    def get_state(self):
        U = np.zeros(5 * self.K * self.n2)
        Bx = np.zeros(self.G)
        By = np.zeros(self.G)
        Bz = np.zeros(self.Z)
        self._L.or_get_state(self._h, U, Bx, By, Bz)
        return U.reshape(5, self.K * self.n2), Bx, By, Bz

    def set_primitive(self, rho, u, p, Bx, By, Bz):
        """Conservative state from nodal primitives (§3.2: m = rho u, E = p/(g-1) + rho|u|^2/2)."""
        rho = np.asarray(rho, dtype=np.float64)
        u = np.asarray(u, dtype=np.float64).reshape(3, -1)
        U = np.zeros((5, rho.size))
        U[0] = rho
        U[1:4] = rho * u
        U[4] = p / (self.gamma - 1.0) + 0.5 * rho * (u ** 2).sum(axis=0)
        self.set_state(U, Bx, By, Bz)

    # -- operators -----------------------------------------------------------
    def hydro_rhs(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64).ravel()
        L = np.zeros_like(U)
        self._L.or_hydro_rhs(self._h, U, L)
        return L.reshape(5, -1)

    def mag_rhs(self, rho, e, u, Bx, By, Bz, eta=None):
        N = self.K * self.n2
        eta = np.zeros(self.K) if eta is None else np.asarray(eta, dtype=np.float64)
        de = np.zeros(N)
        du = np.zeros(3 * N)
        dbx = np.zeros(self.G)
        dby = np.zeros(self.G)
        dbz = np.zeros(self.Z)
        J = np.zeros(3 * self.G)
        E = np.zeros(3 * self.G)
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64).ravel()
        self._L.or_mag_rhs(self._h, f(rho), f(e), f(u), f(Bx), f(By), f(Bz), f(eta), de, du, dbx, dby,
                         dbz, J, E)
        return dict(de=de, du=du.reshape(3, N), dBx=dbx, dBy=dby, dBz=dbz, J=J.reshape(3, -1),
                    E=E.reshape(3, -1))

    def mag_product(self, B, Cb):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64).ravel()
        return self._L.or_mag_product(self._h, *(f(a) for a in B), *(f(a) for a in Cb))

    def hydro_stage_map(self, U, tau):
        U = np.ascontiguousarray(U, dtype=np.float64).ravel().copy()
        self._L.or_hydro_stage_map(self._h, U, tau)
        return U.reshape(5, -1)

    def oe_sensor(self, fields):
        fields = np.ascontiguousarray(fields, dtype=np.float64)
        nc = fields.shape[0]
        s = np.zeros(self.K * 2 * (self.p + 1))
        self._L.or_oe_sensor(self._h, fields.ravel(), nc, s)
        return s.reshape(self.K, 2, self.p + 1)

    def ar_coefficient(self, rho, u, Bx, By, Bz):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64).ravel()
        eta = np.zeros(self.K)
        self._L.or_ar_coefficient(self._h, f(rho), f(u), f(Bx), f(By), f(Bz), eta)
        return eta

    def vel_oe(self, rho, e, u, Bx, By, Bz, tau):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64).ravel()
        e = f(e).copy()
        u = f(u).copy()
        self._L.or_vel_oe(self._h, f(rho), e, u, f(Bx), f(By), f(Bz), tau)
        return e, u.reshape(3, -1)

    # -- stepping ------------------------------------------------------------
    def substep(self, which, tau):
        return self._L.or_substep(self._h, {"H": 0, "M": 1}[which], tau)

    def strang_step(self, dt):
        taken = C.c_double(0.0)
        nrej = C.c_int(0)
        st = self._L.or_strang_step(self._h, dt, C.byref(taken), C.byref(nrej))
        return st, taken.value, nrej.value

    def cfl_dt(self):
        return self._L.or_cfl_dt(self._h)

    def div_metric(self):
        return self._L.or_div_metric(self._h)

    def eta(self):
        out = np.zeros(self.K)
        self._L.or_get_eta(self._h, out)
        return out

    def set_eta(self, eta):
        """Set the element resistivity that :meth:`sample` uses for E_h."""
        self._L.or_set_eta(self._h, np.ascontiguousarray(eta, dtype=np.float64))

    def diagnostics(self):
        out = np.zeros(13)
        self._L.or_diagnostics(self._h, out)
        keys = ["mass", "mom_x", "mom_y", "mom_z", "E_kin", "E_int", "E_mag", "entropy", "div_B",
                "B_max", "rho_min", "p_min", "eta_max"]
        return dict(zip(keys, out))

    FIELDS = {"rho": 0, "mx": 1, "my": 2, "mz": 3, "E": 4, "ux": 5, "uy": 6, "uz": 7, "p": 8,
              "Bx": 9, "By": 10, "Bz": 11, "Ex": 12, "Ey": 13, "Ez": 14, "Jx": 15, "Jy": 16, "Jz": 17}

    def quad_coords(self, nq):
        """Coordinates of the nq x nq Gauss points of every element, [K*nq*nq]."""
        X, Y = np.zeros(self.K * nq * nq), np.zeros(self.K * nq * nq)
        self._L.or_quad_coords(self._h, nq, X, Y)
        return X, Y

    def project_Bz(self, fq, nq):
        """Set B_z to the L2 projection onto V_h^m of values at the points of
        :meth:`quad_coords` (the rest of the state is unchanged)."""
        self._L.or_project_Bz(self._h, np.ascontiguousarray(fq, dtype=np.float64).ravel(), nq)

    def sample(self, field, nq):
        """Values of a field at nq x nq Gauss points per element, with coordinates and weights."""
        size = self.K * nq * nq
        v, X, Y, W = (np.zeros(size) for _ in range(4))
        self._L.or_sample(self._h, self.FIELDS[field], nq, v, X, Y, W)
        return v, X, Y, W


class ParallelOracle(Oracle):
    """The oracle's OpenMP timing build: the same arithmetic with independent
    element loops spread over threads (``set_threads``); used to time the CPU
    baseline on all cores.  Results equal :class:`Oracle`'s bit for bit."""

    @staticmethod
    def _library():
        return omp_lib()

    def set_threads(self, n):
        """Set the thread count (n > 0); returns the count in force."""
        return self._L.or_threads(int(n))


class Tangent(Oracle):
    """The oracle compiled with dual numbers: every map also returns its
    directional derivative (forward mode, exact up to rounding).  Values equal
    those of :class:`Oracle` bit for bit."""

    @staticmethod
    def _library():
        return tangent_lib()

    def set_tangent(self, dU, dBx, dBy, dBz):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64).ravel()
        self._L.or_set_tangent(self._h, f(dU), f(dBx), f(dBy), f(dBz))

    def set_frozen(self, frozen=True):
        """Hold the stabilisation coefficients (OE factors D_l, limiter theta,
        A.R. eta) at their values: the tangent of the frozen-coefficient
        linearisation."""
        self._L.or_set_frozen(self._h, int(frozen))

    def get_tangent(self):
        dU = np.zeros(5 * self.K * self.n2)
        dBx, dBy, dBz = np.zeros(self.G), np.zeros(self.G), np.zeros(self.Z)
        self._L.or_get_tangent(self._h, dU, dBx, dBy, dBz)
        return dU.reshape(5, -1), dBx, dBy, dBz

    def hydro_rhs_tangent(self, U, dU):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64).ravel()
        L = np.zeros(5 * self.K * self.n2)
        dL = np.zeros_like(L)
        self._L.or_hydro_rhs_tangent(self._h, f(U), f(dU), L, dL)
        return L.reshape(5, -1), dL.reshape(5, -1)

    def mag_rhs_tangent(self, state, tangent, eta=None):
        """state / tangent: dicts with rho, e, u [3,N], Bx, By, Bz; returns
        (residual dict, tangent dict) with keys de, du, dBx, dBy, dBz."""
        N = self.K * self.n2
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64).ravel()
        eta = np.zeros(self.K) if eta is None else f(eta)
        keys = ("rho", "e", "u", "Bx", "By", "Bz")
        ins = []
        for k in keys:
            ins += [f(state[k]), f(tangent[k])]
        outs = [np.zeros(N), np.zeros(3 * N), np.zeros(self.G), np.zeros(self.G), np.zeros(self.Z)]
        touts = [np.zeros_like(a) for a in outs]
        self._L.or_mag_rhs_tangent(self._h, *ins, eta, *outs, *touts)
        names = ("de", "du", "dBx", "dBy", "dBz")
        fix = lambda a, n: a.reshape(3, N) if n == "du" else a
        return ({n: fix(a, n) for n, a in zip(names, outs)}, {n: fix(a, n) for n, a in zip(names, touts)})
