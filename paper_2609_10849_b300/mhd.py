"""Thin ctypes binding of libmhd.so (include/mhd.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of the library.  Arrays are numpy (host) or torch CUDA tensors (device,
passed by data pointer on the context's stream).  There is no CPU fallback:
if the library cannot be loaded the import of the solver fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MHD_DEBUG_BUILD=1 selects libmhd_debug.so, the build with index checks
# (mhd_debug_oob); the release library is the default.
LIB_PATH = os.path.join(_HERE, "libmhd_debug.so" if os.environ.get("MHD_DEBUG_BUILD") == "1" else "libmhd.so")

MHD_OK, MHD_RETRIED = 0, 1
MHD_EINVAL, MHD_ENOMEM, MHD_ECUDA, MHD_INADMISSIBLE, MHD_NONFINITE, MHD_TIMEOUT = -1, -2, -3, -4, -5, -6


class MhdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


class Mesh(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double),
                ("y1", C.c_double)]


class Params(C.Structure):
    _fields_ = [("oe_hydro", C.c_int), ("oe_vel", C.c_int), ("pp", C.c_int), ("ar", C.c_int), ("s_H", C.c_double),
                ("s_M", C.c_double), ("C_s", C.c_double), ("C_eta", C.c_double), ("cfl", C.c_double),
                ("max_halvings", C.c_int), ("strang_order", C.c_int), ("reduced_2d2v", C.c_int)]


class Diag(C.Structure):
    _fields_ = [("mass", C.c_double), ("mom", C.c_double * 3), ("E_kin", C.c_double), ("E_int", C.c_double),
                ("E_mag", C.c_double), ("entropy", C.c_double), ("div_B", C.c_double), ("B_max", C.c_double),
                ("rho_min", C.c_double), ("p_min", C.c_double), ("eta_max", C.c_double),
                ("n_rejections", C.c_int), ("stab_active", C.c_int)]


_lib = None

# name: (restype, argtypes); "P" = generic pointer
_SIGS = {
    "mhd_create": (C.c_int, [C.POINTER(Mesh), C.c_int, C.c_int, C.c_double, C.POINTER(C.c_void_p)]),
    "mhd_destroy": (None, [C.c_void_p]),
    "mhd_create_walled": (C.c_int, [C.POINTER(Mesh), C.c_int, C.c_int, C.c_double, C.c_int, C.c_int,
                                    C.POINTER(C.c_void_p)]),
    "mhd_mirror_fill": (C.c_int, [C.c_void_p]),
    "mhd_set_params": (C.c_int, [C.c_void_p, C.POINTER(Params)]),
    "mhd_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mhd_sizes": (C.c_int, [C.c_void_p] + [C.POINTER(C.c_longlong)] * 4),
    "mhd_node_coords": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "mhd_set_state": (C.c_int, [C.c_void_p] + [C.c_void_p] * 4 + [C.c_int]),
    "mhd_get_state": (C.c_int, [C.c_void_p] + [C.c_void_p] * 4 + [C.c_int]),
    "mhd_set_primitive": (C.c_int, [C.c_void_p] + [C.c_void_p] * 3 + [C.c_int]),
    "mhd_primitive_to_conservative": (C.c_int, [C.c_void_p] + [C.c_void_p] * 4 + [C.c_int]),
    "mhd_primitive_to_conservative_vjp": (C.c_int, [C.c_void_p] + [C.c_void_p] * 6 + [C.c_int]),
    "mhd_set_B_from_potential": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_int]),
    "mhd_quad_coords": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "mhd_set_Bz_projected": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "mhd_compute_dt": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "mhd_strang_step": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_double)]),
    "mhd_strang_steps": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int)]),
    "mhd_substep": (C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    "mhd_hydro_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "mhd_mag_rhs": (C.c_int, [C.c_void_p] + [C.c_void_p] * 12 + [C.c_int]),
    "mhd_hydro_stage_map": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_int]),
    "mhd_rcp_check": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]),
    "mhd_sqrt_check": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]),
    "mhd_diagnostics": (C.c_int, [C.c_void_p, C.POINTER(Diag)]),
    "mhd_get_eta": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mhd_launch_count": (C.c_longlong, [C.c_void_p]),
    "mhd_profile_kernels": (C.c_int, [C.c_void_p, C.c_int]),
    "mhd_kernel_times": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "mhd_fp64_peak": (C.c_int, [C.POINTER(C.c_double)]),
    "mhd_hydro_rhs_static": (C.c_int, [C.POINTER(Mesh), C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mhd_batch_create": (C.c_int, [C.c_int, C.POINTER(Mesh), C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.POINTER(C.c_void_p)]),
    "mhd_batch_destroy": (None, [C.c_void_p]),
    "mhd_batch_size": (C.c_int, [C.c_void_p]),
    "mhd_batch_run": (C.c_void_p, [C.c_void_p, C.c_int]),
    "mhd_batch_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "mhd_batch_launch_count": (C.c_longlong, [C.c_void_p]),
    "mhd_state_size": (C.c_longlong, [C.c_void_p]),
    "mhd_adjoint_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                   C.POINTER(C.c_int)]),
    "mhd_adjoint_segment": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                      C.POINTER(C.c_int)]),
    "mhd_hydro_rhs_vjp": (C.c_int, [C.c_void_p] + [C.c_void_p] * 3 + [C.c_int]),
    "mhd_mag_rhs_vjp": (C.c_int, [C.c_void_p] + [C.c_void_p] * 14 + [C.c_int]),
    "mhd_autotune": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mhd_set_tiles": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "mhd_batch_autotune": (C.c_int, [C.c_void_p]),
    "mhd_debug_oob": (C.c_longlong, [C.c_int]),
    "mhd_status_string": (C.c_char_p, [C.c_int]),
    "mhd_last_error": (C.c_char_p, []),
}


def lib():
    """Load libmhd.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing; build it with paper_2609_10849_b300/build.py")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code):
    if code < 0:
        raise MhdError(code, lib().mhd_last_error().decode())
    return code


def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor (float64, contiguous)."""
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous() or str(a.dtype) != "torch.float64":
            raise ValueError("tensors must be contiguous float64")
        return C.c_void_p(a.data_ptr()), int(a.is_cuda)
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise ValueError("arrays must be C-contiguous float64 numpy arrays")
    return a.ctypes.data_as(C.c_void_p), 0


def _ptrs(*arrs):
    ps = [_ptr(a) for a in arrs]
    dev = {d for p, d in ps if p is not None}
    if len(dev) > 1:
        raise ValueError("mix of host and device buffers")
    return [p for p, _ in ps], (dev.pop() if dev else 0)


def fp64_peak_tflops():
    """Measured FP64 FMA issue rate of the current device (TFLOP/s)."""
    v = C.c_double()
    _check(lib().mhd_fp64_peak(C.byref(v)))
    return v.value


def rcp_check(x, y, stream=0):
    """y = the library's FP64 reciprocal of the CUDA tensor x (test hook)."""
    for t in (x, y):
        if not (t.is_cuda and str(t.dtype) == "torch.float64" and t.is_contiguous()):
            raise ValueError("x and y must be contiguous float64 CUDA tensors")
    if x.numel() != y.numel() or x.device != y.device:
        raise ValueError("x and y must have equal size and device")
    _check(lib().mhd_rcp_check(C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), x.numel(), C.c_void_p(stream)))


def sqrt_check(x, y, stream=0):
    """y = the library's FP64 square root of the CUDA tensor x (test hook)."""
    for t in (x, y):
        if not (t.is_cuda and str(t.dtype) == "torch.float64" and t.is_contiguous()):
            raise ValueError("x and y must be contiguous float64 CUDA tensors")
    if x.numel() != y.numel() or x.device != y.device:
        raise ValueError("x and y must have equal size and device")
    _check(lib().mhd_sqrt_check(C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), x.numel(), C.c_void_p(stream)))


def _static_args(nx, ny, p, U, L):
    """Refuse, before anything reaches the library, what the C entry point
    cannot check itself: the C call sees bare device pointers, so a tensor
    shorter than the mesh, one on another GPU than the current one, or an
    output that overlaps the input would make its kernels read or write
    outside the caller's buffers (or break their no-alias contract)."""
    need = 5 * int(nx) * int(ny) * (int(p) + 1) ** 2
    for name, t in (("U", U), ("L", L)):
        if not hasattr(t, "data_ptr"):
            raise ValueError(f"{name} must be a torch tensor")
        if str(t.dtype) != "torch.float64" or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 tensor")
        if t.numel() != need:
            raise ValueError(f"{name} has {t.numel()} entries; the mesh needs 5 K (p+1)^2 = {need}")
    u0, l0 = U.data_ptr(), L.data_ptr()
    if u0 < l0 + 8 * need and l0 < u0 + 8 * need:
        raise ValueError("L must not overlap U")
    if not (U.is_cuda and L.is_cuda):
        raise ValueError("U and L must be CUDA tensors")
    import torch
    cur = torch.cuda.current_device()
    if U.device.index != cur or L.device.index != cur:
        raise ValueError(f"U and L must be on the current device cuda:{cur}")


def hydro_rhs_static(nx, ny, p, gamma, domain, U, L, stream=0):
    """Hydro residual of the device tensor U [5, K (p+1)^2] into the device
    tensor L without any device allocation (fixed library scratch; calls that
    overlap on the GPU race).  Enqueued on `stream`; does not synchronise.
    Sizes, device and aliasing are checked here first (ValueError)."""
    _static_args(nx, ny, p, U, L)
    mesh = Mesh(nx, ny, *(float(v) for v in domain))
    _check(lib().mhd_hydro_rhs_static(C.byref(mesh), p, float(gamma), C.c_void_p(U.data_ptr()),
                                      C.c_void_p(L.data_ptr()), C.c_void_p(stream)))


class Solver:
    """One periodic mesh with DGSEM degree p and magnetic degree k."""

    def __init__(self, nx, ny, p, k, gamma, domain=(0.0, 1.0, 0.0, 1.0), _handle=None, walls=0, conducting=0):
        """walls (bit 0 x, bit 1 y) != 0: reflecting walls on the physical
        domain by the method of images (mhd_create_walled); the solver then
        holds the doubled periodic mesh (nx, ny, domain and every layout are
        the doubled ones; the physical elements are those of ``physical``)."""
        self.p, self.k, self.gamma = p, k, gamma
        self.walls, self.conducting = walls, conducting
        self._owned = _handle is None
        x0, x1, y0, y1 = (float(v) for v in domain)
        self.physical = (nx, ny, (x0, x1, y0, y1))
        if walls & 1:
            nx, x1 = 2 * nx, 2.0 * x1 - x0
        if walls & 2:
            ny, y1 = 2 * ny, 2.0 * y1 - y0
        self.nx, self.ny, self.domain = nx, ny, (x0, x1, y0, y1)
        if _handle is None:
            h = C.c_void_p()
            if walls:
                mesh = Mesh(*self.physical[:2], *self.physical[2])
                _check(lib().mhd_create_walled(C.byref(mesh), p, k, gamma, int(walls), int(conducting), C.byref(h)))
            else:
                mesh = Mesh(nx, ny, *self.domain)
                _check(lib().mhd_create(C.byref(mesh), p, k, gamma, C.byref(h)))
        else:
            h = C.c_void_p(_handle)
        self._h = h
        K, N, G, Z = (C.c_longlong() for _ in range(4))
        _check(lib().mhd_sizes(h, C.byref(K), C.byref(N), C.byref(G), C.byref(Z)))
        self.K, self.N, self.G, self.Z = K.value, N.value, G.value, Z.value
        self.params = dict(oe_hydro=0, oe_vel=0, pp=0, ar=0, s_H=0.02, s_M=0.02, C_s=5.0, C_eta=0.2, cfl=0.4,
                           max_halvings=20, strang_order=0, reduced_2d2v=0)

    def close(self):
        if getattr(self, "_h", None):
            if self._owned:
                lib().mhd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def mirror_fill(self):
        """Write the images of the physical part (walled solvers)."""
        _check(lib().mhd_mirror_fill(self._h))

    def set_params(self, **kw):
        """Update stabilisation / stepping parameters; on MHD_EINVAL the previous
        parameters stay in force (here and in the library)."""
        new = dict(self.params, **kw)
        _check(lib().mhd_set_params(self._h, C.byref(Params(**new))))
        self.params = new

    def set_stream(self, stream_ptr: int):
        _check(lib().mhd_set_stream(self._h, C.c_void_p(stream_ptr)))

    def coords(self, which):
        size = {"dg": self.N, "w": self.G, "bz": self.Z}[which]
        X, Y = np.zeros(size), np.zeros(size)
        _check(lib().mhd_node_coords(self._h, {"dg": 0, "w": 1, "bz": 2}[which], _ptr(X)[0], _ptr(Y)[0]))
        return X, Y

    def set_state(self, U, Bx, By, Bz):
        (pU, pX, pY, pZ), dev = _ptrs(U, Bx, By, Bz)
        _check(lib().mhd_set_state(self._h, pU, pX, pY, pZ, dev))

    def get_state(self, out=None):
        if out is None:
            out = (np.zeros((5, self.N)), np.zeros(self.G), np.zeros(self.G), np.zeros(self.Z))
        (pU, pX, pY, pZ), dev = _ptrs(*out)
        _check(lib().mhd_get_state(self._h, pU, pX, pY, pZ, dev))
        return out

    def set_primitive(self, rho, u, p):
        (a, b, c), dev = _ptrs(rho, u, p)
        _check(lib().mhd_set_primitive(self._h, a, b, c, dev))

    def primitive_to_conservative(self, rho, u, p, out):
        """U [5, N] = (rho, rho u, p/(gamma-1) + rho|u|^2/2) into ``out``
        (numpy arrays or CUDA tensors); the solver's state is not touched."""
        (a, b, c, o), dev = _ptrs(rho, u, p, out)
        _check(lib().mhd_primitive_to_conservative(self._h, a, b, c, o, dev))
        return out

    def primitive_to_conservative_vjp(self, rho, u, lamU, g_rho, g_u, g_p):
        """dJ/d(rho, u, p) from lamU = dJ/dU at (rho, u), into the given buffers."""
        ps, dev = _ptrs(rho, u, lamU, g_rho, g_u, g_p)
        _check(lib().mhd_primitive_to_conservative_vjp(self._h, *ps, dev))
        return g_rho, g_u, g_p

    def set_B_from_potential(self, Az, Bx0, By0, Bz):
        (a, z), dev = _ptrs(Az, Bz)
        _check(lib().mhd_set_B_from_potential(self._h, a, float(Bx0), float(By0), z, dev))

    def quad_coords(self, nq):
        """Coordinates of the nq x nq Gauss points of every element, [K*nq*nq]."""
        size = self.K * nq * nq
        X, Y = np.zeros(size), np.zeros(size)
        _check(lib().mhd_quad_coords(self._h, int(nq), _ptr(X)[0], _ptr(Y)[0]))
        return X, Y

    def set_Bz_projected(self, fq, nq):
        """B_z as the L2 projection onto V_h^k of values at :meth:`quad_coords`."""
        (a,), dev = _ptrs(fq)
        _check(lib().mhd_set_Bz_projected(self._h, a, int(nq), dev))

    def compute_dt(self):
        dt = C.c_double()
        _check(lib().mhd_compute_dt(self._h, C.byref(dt)))
        return dt.value

    def strang_step(self, dt=0.0):
        taken = C.c_double()
        st = _check(lib().mhd_strang_step(self._h, float(dt), C.byref(taken)))
        return st, taken.value

    def strang_steps(self, dt, nsteps):
        done = C.c_int()
        _check(lib().mhd_strang_steps(self._h, float(dt), int(nsteps), C.byref(done)))
        return done.value

    def substep(self, which, tau):
        return _check(lib().mhd_substep(self._h, {"H": 0, "M": 1}[which], float(tau)))

    def hydro_rhs(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        L = np.zeros_like(U)
        _check(lib().mhd_hydro_rhs(self._h, _ptr(U)[0], _ptr(L)[0], 0))
        return L

    def hydro_stage_map(self, U, tau):
        """Stage map P = P_PP o P_OE of the enabled maps on a conservative state."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        out = np.zeros_like(U)
        _check(lib().mhd_hydro_stage_map(self._h, _ptr(U)[0], float(tau), _ptr(out)[0], 0))
        return out

    def mag_rhs(self, rho, e, u, Bx, By, Bz, eta=None):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        eta = np.zeros(self.K) if eta is None else eta
        ins = [f(a) for a in (rho, e, u, Bx, By, Bz, eta)]
        de, du = np.zeros(self.N), np.zeros((3, self.N))
        dBx, dBy, dBz = np.zeros(self.G), np.zeros(self.G), np.zeros(self.Z)
        ps = [_ptr(a)[0] for a in ins + [de, du, dBx, dBy, dBz]]
        _check(lib().mhd_mag_rhs(self._h, *ps, 0))
        return dict(de=de, du=du, dBx=dBx, dBy=dBy, dBz=dBz)

    # -- tiles ---------------------------------------------------------------
    def autotune(self):
        """Time the elements-per-CTA variants on the current state and keep the
        fastest; returns (volume elements per CTA, magnetic elements per CTA)."""
        ch = np.zeros(2, dtype=np.int32)
        _check(lib().mhd_autotune(self._h, ch.ctypes.data_as(C.c_void_p)))
        return int(ch[0]), int(ch[1])

    def set_tiles(self, vol_variant, mag_variant):
        _check(lib().mhd_set_tiles(self._h, int(vol_variant), int(mag_variant)))

    # -- packed state and adjoint ------------------------------------------
    def state_size(self):
        """Length of the packed state [U 5N | Bx G | By G | Bz Z] (host layouts)."""
        return int(lib().mhd_state_size(self._h))

    def _split(self, x):
        N5, G, Z = 5 * self.N, self.G, self.Z
        return x[:N5], x[N5:N5 + G], x[N5 + G:N5 + 2 * G], x[N5 + 2 * G:N5 + 2 * G + Z]

    def set_packed(self, x):
        """Set the state from a packed vector (numpy array or CUDA tensor)."""
        self.set_state(*self._split(x))

    def get_packed(self, out):
        """Write the packed state into ``out`` (numpy array or CUDA tensor)."""
        self.get_state(self._split(out))
        return out

    def adjoint_step(self, state, lam, dt, out=None):
        """lam_n = (dS^dt/dx)(state)^T lam for one Strang step at fixed dt.

        ``state``, ``lam`` and ``out`` are packed vectors, all numpy arrays or
        all CUDA tensors; ``out`` may be ``lam``."""
        if out is None:
            out = np.zeros_like(lam) if isinstance(lam, np.ndarray) else lam.clone()
        (ps, pl, po), dev = _ptrs(state, lam, out)
        flags = C.c_int(0)
        code = lib().mhd_adjoint_step(self._h, ps, pl, po, float(dt), dev, C.byref(flags))
        self.last_adjoint_flags = flags.value  # stabilisation maps differentiated with frozen coefficients
        if code < 0:
            raise MhdError(code, lib().mhd_last_error().decode() + f" (flags {flags.value})")
        return out

    def adjoint_segment(self, state, nsteps, lam, dt, out=None):
        """lam_0 for nsteps fixed-dt steps from ``state`` (one checkpoint segment,
        recorded in device memory in one forward pass); ``out`` may be ``lam``."""
        if out is None:
            out = np.zeros_like(lam) if isinstance(lam, np.ndarray) else lam.clone()
        (ps, pl, po), dev = _ptrs(state, lam, out)
        flags = C.c_int(0)
        code = lib().mhd_adjoint_segment(self._h, ps, int(nsteps), pl, po, float(dt), dev, C.byref(flags))
        self.last_adjoint_flags = flags.value
        if code < 0:
            raise MhdError(code, lib().mhd_last_error().decode() + f" (flags {flags.value})")
        return out

    def hydro_rhs_vjp(self, U, nu):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        U, nu = f(U), f(nu)
        out = np.zeros_like(U)
        _check(lib().mhd_hydro_rhs_vjp(self._h, _ptr(U)[0], _ptr(nu)[0], _ptr(out)[0], 0))
        return out

    def mag_rhs_vjp(self, rho, u, Bx, By, Bz, w_u, w_Bx, w_By, w_Bz):
        """VJP of the ideal magnetic residual: returns g_rho, g_u [3,N], g_Bx, g_By, g_Bz."""
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        ins = [f(a) for a in (rho, u, Bx, By, Bz, w_u, w_Bx, w_By, w_Bz)]
        outs = [np.zeros(self.N), np.zeros((3, self.N)), np.zeros(self.G), np.zeros(self.G), np.zeros(self.Z)]
        _check(lib().mhd_mag_rhs_vjp(self._h, *[_ptr(a)[0] for a in ins + outs], 0))
        return outs

    def diagnostics(self):
        d = Diag()
        _check(lib().mhd_diagnostics(self._h, C.byref(d)))
        return dict(mass=d.mass, mom_x=d.mom[0], mom_y=d.mom[1], mom_z=d.mom[2], E_kin=d.E_kin, E_int=d.E_int,
                    E_mag=d.E_mag, entropy=d.entropy, div_B=d.div_B, B_max=d.B_max, rho_min=d.rho_min,
                    p_min=d.p_min, eta_max=d.eta_max, n_rejections=d.n_rejections, stab_active=d.stab_active)

    def eta(self):
        out = np.zeros(self.K)
        _check(lib().mhd_get_eta(self._h, _ptr(out)[0]))
        return out

    def launch_count(self):
        return lib().mhd_launch_count(self._h)

    KERNEL_CLASSES = ("face", "vol", "mag_J", "mag_stage", "mag_B", "exchange", "stab_hydro", "stab_eta",
                      "stab_vel")

    def profile_kernels(self, enable=True):
        _check(lib().mhd_profile_kernels(self._h, int(enable)))

    def kernel_times(self):
        """{class: (total ms, launch groups)} since profiling was enabled."""
        n = len(self.KERNEL_CLASSES)
        ms = np.zeros(n)
        cnt = np.zeros(n, dtype=np.int64)
        _check(lib().mhd_kernel_times(self._h, ms.ctypes.data_as(C.c_void_p), cnt.ctypes.data_as(C.c_void_p), n))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(self.KERNEL_CLASSES) if cnt[i]}


class Batch:
    """Independent runs advanced together by one CUDA-graph launch per call.

    ``specs`` is a list of (nx, ny, p, k, gamma, domain); ``runs[i]`` is a
    :class:`Solver` view of run i (owned by the batch)."""

    def __init__(self, specs):
        n = len(specs)
        meshes = (Mesh * n)(*[Mesh(s[0], s[1], *(float(v) for v in s[5])) for s in specs])
        p = np.array([s[2] for s in specs], dtype=np.int32)
        k = np.array([s[3] for s in specs], dtype=np.int32)
        g = np.array([s[4] for s in specs], dtype=np.float64)
        h = C.c_void_p()
        _check(lib().mhd_batch_create(n, meshes, p.ctypes.data_as(C.c_void_p), k.ctypes.data_as(C.c_void_p),
                                      g.ctypes.data_as(C.c_void_p), C.byref(h)))
        self._h = h
        self.runs = [Solver(s[0], s[1], s[2], s[3], s[4], s[5], _handle=lib().mhd_batch_run(h, i))
                     for i, s in enumerate(specs)]

    def step(self, dt, nsteps=1):
        """Advance every run by nsteps Strang steps of its own dt; returns per-run status."""
        dt = np.ascontiguousarray(dt, dtype=np.float64)
        st = np.zeros(len(self.runs), dtype=np.int32)
        code = lib().mhd_batch_step(self._h, dt.ctypes.data_as(C.c_void_p), int(nsteps), st.ctypes.data_as(C.c_void_p))
        if code < 0 and code != MHD_INADMISSIBLE:
            raise MhdError(code, lib().mhd_last_error().decode())
        return st

    def launch_count(self):
        return lib().mhd_batch_launch_count(self._h)

    def autotune(self):
        """Autotune the tiles of every run (each run keeps its own choice)."""
        _check(lib().mhd_batch_autotune(self._h))

    def close(self):
        if getattr(self, "_h", None):
            for r in self.runs:
                r._h = None
            lib().mhd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
