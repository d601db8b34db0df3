"""FP64 CPU oracle for the registration objective of arXiv 1807.00467, Sec. II-D.

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg are the only users.  It shares no code with
the GPU library (``paper_1807_00467_gb300``) and is never a fallback for it.

The C sources (``ngf_oracle.c``) are compiled with gcc into
``oracle/libngf_oracle.so`` by :func:`build`; this module wraps them with
numpy arrays.  Images are float32 ``[nz][ny][nx]``; grid fields are float64
``[3][mz][my][mx]`` (mm).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ngf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libngf_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction)."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                                  os.path.getmtime(os.path.join(_HERE, "ngf_oracle.h"))))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double * 3), ("m", C.c_int * 3),
                ("R", C.POINTER(C.c_float)), ("T", C.POINTER(C.c_float)),
                ("eta", C.c_double), ("alpha", C.c_double), ("gamma", C.c_double),
                ("delta", C.c_double), ("nk", C.c_int),
                ("kx", C.POINTER(C.c_double)), ("ky", C.POINTER(C.c_double))]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.POINTER(_Problem)
        dp = C.POINTER(C.c_double)
        fp = C.POINTER(C.c_float)
        ip = C.POINTER(C.c_int)
        L.orc_check.argtypes = [P]
        L.orc_prolong.argtypes = [P, dp, dp]
        L.orc_warp.argtypes = [P, dp, dp, dp]
        L.orc_cells.argtypes = [P, dp, ip]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_ngf_distance.argtypes = [P, dp, dp, dp]
        L.orc_ngf_distance.restype = C.c_double
        L.orc_objective.argtypes = [P, dp, dp]
        L.orc_gradient.argtypes = [P, dp, dp, dp]
        L.orc_ngf_gradient.argtypes = [P, dp, dp, dp]
        L.orc_curvature.argtypes = [P, dp, dp, dp, dp]
        L.orc_vcc.argtypes = [P, dp, dp, dp, dp, dp]
        L.orc_keypoints.argtypes = [P, dp, dp, dp, dp]
        L.orc_vcc_cell_dets.argtypes = [P, dp, ip, dp]
        L.orc_linearize.argtypes = [P, dp]
        L.orc_linearize.restype = C.c_void_p
        L.orc_lin_free.argtypes = [C.c_void_p]
        L.orc_ngf_gn_matvec.argtypes = [P, C.c_void_p, dp, dp]
        L.orc_gn_matvec.argtypes = [P, C.c_void_p, dp, dp]
        L.orc_gn_diag.argtypes = [P, C.c_void_p, C.c_double, dp]
        L.orc_vcc_diag.argtypes = [P, dp, dp]
        L.orc_pcg.argtypes = [P, C.c_void_p, dp, dp, C.c_int, C.c_double, dp]
        L.orc_gn_solve.argtypes = [P, dp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, dp]
        L.orc_restrict_image.argtypes = [ip, fp, fp]
        L.orc_prolong_grid.argtypes = [ip, dp, ip, dp]
        L.orc_register_pyramid.argtypes = [P, C.c_int, dp, C.c_int, C.c_int, C.c_int, C.c_double,
                                           C.c_double, C.c_int, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """One registration problem: images, spacing, grid, weights, keypoints."""

    def __init__(self, R, T, h, m, eta=10.0, alpha=1.0, gamma=0.0, delta=0.0, kx=None, ky=None):
        self.R = np.ascontiguousarray(R, dtype=np.float32)
        self.T = np.ascontiguousarray(T, dtype=np.float32)
        assert self.R.shape == self.T.shape
        self.n = (self.R.shape[2], self.R.shape[1], self.R.shape[0])
        self.h = tuple(float(v) for v in h)
        self.m = tuple(int(v) for v in m)
        self.kx = None if kx is None else _f64(kx).reshape(-1, 3)
        self.ky = None if ky is None else _f64(ky).reshape(-1, 3)
        self.s = _Problem()
        self.s.n[:] = self.n
        self.s.h[:] = self.h
        self.s.m[:] = self.m
        self.s.R = self.R.ctypes.data_as(C.POINTER(C.c_float))
        self.s.T = self.T.ctypes.data_as(C.POINTER(C.c_float))
        self.s.eta, self.s.alpha, self.s.gamma, self.s.delta = eta, alpha, gamma, delta
        if self.kx is not None:
            self.s.nk = len(self.kx)
            self.s.kx = _dp(self.kx)
            self.s.ky = _dp(self.ky)
        if lib().orc_check(C.byref(self.s)) != 0:
            raise ValueError(f"invalid oracle problem n={self.n} m={self.m}")

    @property
    def delta(self):
        return self.s.delta

    @delta.setter
    def delta(self, v):
        self.s.delta = float(v)

    @property
    def grid_shape(self):
        return (3, self.m[2], self.m[1], self.m[0])

    @property
    def N(self):
        return self.n[0] * self.n[1] * self.n[2]

    def _ref(self):
        return C.byref(self.s)

    def prolong(self, u):
        u = _f64(u)
        out = np.empty((3, self.n[2], self.n[1], self.n[0]))
        lib().orc_prolong(self._ref(), _dp(u), _dp(out))
        return out

    def cells(self, u):
        """Sample cell per voxel and axis (int32 [3][nz][ny][nx]) as decided in FP32."""
        u = _f64(u)
        k = np.empty((3, self.n[2], self.n[1], self.n[0]), dtype=np.int32)
        lib().orc_cells(self._ref(), _dp(u), k.ctypes.data_as(C.POINTER(C.c_int)))
        return k

    def warp(self, u):
        u = _f64(u)
        Tw = np.empty((self.n[2], self.n[1], self.n[0]))
        dT = np.empty((3,) + Tw.shape)
        lib().orc_warp(self._ref(), _dp(u), _dp(Tw), _dp(dT))
        return Tw, dT

    def ngf_distance(self, Tw):
        Tw = _f64(Tw)
        r = np.empty_like(Tw)
        a = np.empty((3,) + Tw.shape)
        D = lib().orc_ngf_distance(self._ref(), _dp(Tw), _dp(r), _dp(a))
        return D, r, a

    def objective(self, u):
        u = _f64(u)
        terms = np.zeros(5)
        st = lib().orc_objective(self._ref(), _dp(u), _dp(terms))
        return terms, st

    def gradient(self, u):
        u = _f64(u)
        terms = np.zeros(5)
        g = np.zeros(self.grid_shape)
        st = lib().orc_gradient(self._ref(), _dp(u), _dp(terms), _dp(g))
        return terms, g, st

    def ngf_gradient(self, u):
        u = _f64(u)
        D = C.c_double()
        g = np.zeros(self.grid_shape)
        lib().orc_ngf_gradient(self._ref(), _dp(u), C.byref(D), _dp(g))
        return D.value, g

    def curvature(self, u, v=None):
        u = _f64(u)
        e = C.c_double()
        out = np.zeros(self.grid_shape)
        vv = None if v is None else _f64(v)
        lib().orc_curvature(self._ref(), _dp(u), None if vv is None else _dp(vv), C.byref(e), _dp(out))
        return e.value, out

    def vcc(self, u, v=None):
        u = _f64(u)
        e = C.c_double()
        out = np.zeros(self.grid_shape)
        mm = np.zeros(2)
        vv = None if v is None else _f64(v)
        st = lib().orc_vcc(self._ref(), _dp(u), None if vv is None else _dp(vv), C.byref(e), _dp(out), _dp(mm))
        return e.value, out, st, (mm[0], mm[1])

    def vcc_cell_dets(self, u, cell):
        u = _f64(u)
        d = np.zeros(64)
        c = (C.c_int * 3)(*cell)
        lib().orc_vcc_cell_dets(self._ref(), _dp(u), c, _dp(d))
        return d.reshape(4, 4, 4).transpose(2, 1, 0)    # [a][b][c]

    def keypoints(self, u, v=None):
        u = _f64(u)
        e = C.c_double()
        out = np.zeros(self.grid_shape)
        vv = None if v is None else _f64(v)
        lib().orc_keypoints(self._ref(), _dp(u), None if vv is None else _dp(vv), C.byref(e), _dp(out))
        return e.value, out

    def linearize(self, u):
        return Lin(self, u)

    def vcc_diag(self, u):
        u = _f64(u)
        d = np.zeros(self.grid_shape)
        lib().orc_vcc_diag(self._ref(), _dp(u), _dp(d))
        return d

    def gn_solve(self, u0, gn_iters, pcg_iters, ls_max=10, armijo_c=1e-4, tau=0.0, delta_adaptive=False):
        u = _f64(u0).copy()
        rep = np.zeros((gn_iters, 8))
        st = lib().orc_gn_solve(self._ref(), _dp(u), gn_iters, pcg_iters, ls_max, armijo_c, tau,
                                int(delta_adaptive), _dp(rep))
        return u, rep, st

    def register_pyramid(self, u0, levels, gn_iters, pcg_iters, ls_max=10, armijo_c=1e-4, tau=0.0,
                         delta_adaptive=False):
        u = _f64(u0).copy()
        rep = np.zeros((levels, gn_iters, 8))
        st = lib().orc_register_pyramid(self._ref(), levels, _dp(u), gn_iters, pcg_iters, ls_max,
                                        armijo_c, tau, int(delta_adaptive), _dp(rep))
        return u, rep, st


class Lin:
    """Stored Gauss-Newton linearisation at u."""

    def __init__(self, prob: Problem, u):
        self.prob = prob
        self.u = _f64(u)
        self.ptr = lib().orc_linearize(prob._ref(), _dp(self.u))

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().orc_lin_free(self.ptr)
            self.ptr = None

    def ngf_matvec(self, v):
        v = _f64(v)
        out = np.zeros(self.prob.grid_shape)
        lib().orc_ngf_gn_matvec(self.prob._ref(), self.ptr, _dp(v), _dp(out))
        return out

    def matvec(self, v):
        v = _f64(v)
        out = np.zeros(self.prob.grid_shape)
        lib().orc_gn_matvec(self.prob._ref(), self.ptr, _dp(v), _dp(out))
        return out

    def gn_diag(self, tau=0.0):
        d = np.zeros(self.prob.grid_shape)
        lib().orc_gn_diag(self.prob._ref(), self.ptr, tau, _dp(d))
        return d

    def pcg(self, g, iters, tau=0.0):
        g = _f64(g)
        s = np.zeros(self.prob.grid_shape)
        stats = np.zeros(3)
        lib().orc_pcg(self.prob._ref(), self.ptr, _dp(g), _dp(s), iters, tau, _dp(stats))
        return s, stats


def restrict_image(img):
    img = np.ascontiguousarray(img, dtype=np.float32)
    n = (C.c_int * 3)(img.shape[2], img.shape[1], img.shape[0])
    out = np.empty((img.shape[0] // 2, img.shape[1] // 2, img.shape[2] // 2), dtype=np.float32)
    lib().orc_restrict_image(n, img.ctypes.data_as(C.POINTER(C.c_float)), out.ctypes.data_as(C.POINTER(C.c_float)))
    return out


def prolong_grid(uc, mf):
    uc = _f64(uc)
    mc = (C.c_int * 3)(uc.shape[3], uc.shape[2], uc.shape[1])
    mfa = (C.c_int * 3)(*mf)
    out = np.empty((3, mf[2], mf[1], mf[0]))
    lib().orc_prolong_grid(mc, _dp(uc), mfa, _dp(out))
    return out


def num_threads():
    return lib().orc_num_threads()


def set_threads(n):
    """OpenMP threads of later oracle calls in this process."""
    lib().orc_set_threads(int(n))
