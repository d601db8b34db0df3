"""Python binding of the ngfreg C ABI over torch CUDA tensors.

Every function marshals tensors into pointers and calls the entry point of
the same name in libngfreg.so; all arithmetic runs in the library's kernels.
PyTorch provides device memory (including the context workspace) and streams.

Shapes: images (nz, ny, nx) float32 (or float16 holding HU + 1024), grid
fields (3, mz, my, mx) float32 in mm, keypoints (nk, 3) float32 in mm, terms
(5,) float64 = (D, R, V, K, J) of Eq. (11).
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import (RG_CURV, RG_EFOLD, RG_F16, RG_F32, RG_KP, RG_OK, RG_REPORT_COLS, RG_VCC, GridGeom, ImageGeom,
                   NgfError, Params, Schedule)

__all__ = ["Context", "register_pyramid", "restrict_image", "prolong_grid", "launch_count", "RG_CURV", "RG_VCC", "RG_KP",
           "RG_EFOLD", "NgfError", "make_params", "make_schedule"]


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _stream_ptr(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _check(code, ctx=None, name=""):
    if code < 0:
        msg = _lib.load().rg_last_error(ctx).decode() if ctx else ""
        raise NgfError(code, f"{name}: {msg}")
    return code


def make_params(eta=10.0, alpha=1.0, gamma=0.0, delta=0.0, delta_adaptive=False, tau=0.0, det_lo=0.25, det_hi=4.0):
    """det_lo, det_hi: reporting bounds on the Jacobian bounds d (report column 10)."""
    return Params(eta, alpha, gamma, delta, int(bool(delta_adaptive)), tau, det_lo, det_hi)


SCHED_DEVICE, SCHED_GRAPH, SCHED_AUTOTUNE = 1, 2, 4    # rg_schedule.flags


def make_schedule(levels=1, gn_iters=5, pcg_iters=30, ls_max=10, armijo_c=1e-4, drive="host", autotune=False):
    """drive: 'host' (line search read on the host), 'device' (decided on the
    GPU, no per-iteration synchronisation) or 'graph' (device, with each
    iteration replayed from a captured CUDA graph); autotune: pick each
    level's tile shape with rg_autotune first."""
    flags = {"host": 0, "device": SCHED_DEVICE, "graph": SCHED_GRAPH}[drive] | (SCHED_AUTOTUNE if autotune else 0)
    return Schedule(levels, gn_iters, pcg_iters, ls_max, armijo_c, flags)


def _img_geom(shape, h):
    g = ImageGeom()
    g.n[:] = (shape[2], shape[1], shape[0])
    g.h[:] = tuple(float(v) for v in h)
    return g


def _grid_geom(m):
    g = GridGeom()
    g.m[:] = tuple(int(v) for v in m)
    return g


def _dtype_code(t):
    if t.dtype == torch.float32:
        return RG_F32
    if t.dtype == torch.float16:
        return RG_F16
    raise TypeError(f"images must be float32 or float16, got {t.dtype}")


class Context:
    """A registration problem bound to device images and a workspace."""

    def __init__(self, R, T, h, m, params=None, nk_max=0, stream=None, pcg_max=30):
        L = _lib.load()
        if not (R.is_cuda and T.is_cuda and R.shape == T.shape and R.dtype == T.dtype and R.dim() == 3):
            raise ValueError("R, T must be CUDA tensors of equal shape (nz, ny, nx) and dtype")
        self.R, self.T = R.contiguous(), T.contiguous()
        self.dtype = _dtype_code(self.R)
        self.h = tuple(float(v) for v in h)
        self.m = tuple(int(v) for v in m)
        self.n = (R.shape[2], R.shape[1], R.shape[0])
        self.ig, self.gg = _img_geom(R.shape, h), _grid_geom(m)
        self.params = params if params is not None else make_params()
        self.nk_max = int(nk_max)
        self.pcg_max = int(pcg_max)
        self.stream = stream
        nbytes = C.c_size_t()
        _check(L.rg_workspace_size(C.byref(self.ig), C.byref(self.gg), self.dtype, self.nk_max, self.pcg_max,
                                   C.byref(nbytes)), name="rg_workspace_size")
        self.workspace = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=R.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        self._ctx = C.c_void_p()
        _check(L.rg_ctx_create(C.byref(self._ctx), C.byref(self.ig), C.byref(self.gg), self.dtype,
                               C.byref(self.params), self.nk_max, self.pcg_max, C.c_void_p(self._ws_ptr), nbytes.value,
                               _stream_ptr(stream)), name="rg_ctx_create")
        _check(L.rg_set_images(self._ctx, _ptr(self.R), _ptr(self.T)), self._ctx, "rg_set_images")
        self.kx = self.ky = None
        self.nk = 0
        self.device = R.device

    # -- helpers
    def __del__(self):
        if getattr(self, "_ctx", None):
            _lib.load().rg_ctx_destroy(self._ctx)
            self._ctx = None

    @property
    def grid_shape(self):
        return (3, self.m[2], self.m[1], self.m[0])

    def _field(self, x):
        if not (x.is_cuda and x.dtype == torch.float32 and tuple(x.shape) == self.grid_shape and x.is_contiguous()):
            raise ValueError(f"grid field must be a contiguous float32 CUDA tensor of shape {self.grid_shape}")
        return x

    def _new_field(self):
        return torch.empty(self.grid_shape, dtype=torch.float32, device=self.device)

    def _terms(self):
        return torch.empty(5, dtype=torch.float64, device=self.device)

    # -- entry points
    def set_params(self, params):
        self.params = params
        _check(_lib.load().rg_set_params(self._ctx, C.byref(params)), self._ctx, "rg_set_params")

    def get_params(self):
        p = Params()
        _lib.load().rg_get_params(self._ctx, C.byref(p))
        return p

    def set_tile(self, tile_y):
        """Tile height (8 or 16 voxel rows) of the NGF kernels (tuning)."""
        _check(_lib.load().rg_set_tile(self._ctx, int(tile_y)), self._ctx, "rg_set_tile")

    def autotune(self, u):
        """Times the kernel candidates at u and keeps the fastest; returns
        (tile_y, general): general 1 for the general kernels, 2 / 3 for the
        specialised kernels with the column / tile objective-gradient pass
        (include/ngfreg.h, rg_autotune).  Discards the linearisation."""
        ty, gen = C.c_int32(), C.c_int32()
        _check(_lib.load().rg_autotune(self._ctx, _ptr(self._field(u)), C.byref(ty), C.byref(gen)), self._ctx,
               "rg_autotune")
        return ty.value, gen.value

    def set_keypoints(self, kx, ky):
        kx = kx.contiguous().float()
        ky = ky.contiguous().float()
        self.kx, self.ky, self.nk = kx, ky, int(kx.shape[0])
        _check(_lib.load().rg_set_keypoints(self._ctx, self.nk, _ptr(kx), _ptr(ky)), self._ctx, "rg_set_keypoints")

    def ngf_objective(self, u, terms=None):
        terms = self._terms() if terms is None else terms
        code = _check(_lib.load().ngf_objective(self._ctx, _ptr(self._field(u)), _ptr(terms)), self._ctx,
                      "ngf_objective")
        return terms

    def ngf_gradient(self, u, grad=None, terms=None):
        terms = self._terms() if terms is None else terms
        grad = self._new_field() if grad is None else grad
        _check(_lib.load().ngf_gradient(self._ctx, _ptr(self._field(u)), _ptr(terms), _ptr(grad)), self._ctx,
               "ngf_gradient")
        return terms, grad

    def gn_linearize(self, u, want_grad=True):
        terms = self._terms()
        grad = self._new_field() if want_grad else None
        _check(_lib.load().gn_linearize(self._ctx, _ptr(self._field(u)), _ptr(terms), _ptr(grad)), self._ctx,
               "gn_linearize")
        return terms, grad

    def gn_matvec(self, v, out=None):
        out = self._new_field() if out is None else out
        _check(_lib.load().gn_matvec(self._ctx, _ptr(self._field(v)), _ptr(out)), self._ctx, "gn_matvec")
        return out

    def regularizer_apply(self, which, u, v=None):
        energy = torch.empty(1, dtype=torch.float64, device=self.device)
        out = self._new_field()
        _check(_lib.load().regularizer_apply(self._ctx, int(which), _ptr(self._field(u)),
                                             _ptr(None if v is None else self._field(v)), _ptr(energy), _ptr(out)),
               self._ctx, "regularizer_apply")
        return energy, out

    def gn_pcg_solve(self, g, iters, p=None):
        p = self._new_field() if p is None else p
        stats = torch.empty(3, dtype=torch.float64, device=self.device)
        _check(_lib.load().gn_pcg_solve(self._ctx, _ptr(self._field(g)), _ptr(p), int(iters), _ptr(stats)),
               self._ctx, "gn_pcg_solve")
        return p, stats

    def sync(self):
        """Synchronises the context stream; returns the latched device status
        (RG_OK) or raises NgfError with RG_ETIMEOUT / RG_ENONFINITE."""
        return _check(_lib.load().rg_sync(self._ctx), self._ctx, "rg_sync")

    def debug_hook(self, what, value):
        """Test hooks of include/ngfreg.h (RG_HOOK_NO_TMA, RG_HOOK_POLL_LIMIT, RG_HOOK_PASS)."""
        _check(_lib.load().rg_debug_hook(self._ctx, int(what), int(value)), self._ctx, "rg_debug_hook")

    def profile(self, enable=True):
        """Record CUDA events around every kernel launch on the context stream."""
        _check(_lib.load().rg_profile(self._ctx, int(bool(enable))), self._ctx, "rg_profile")

    def profile_read(self, kernel):
        """(total ms, launches) of one kernel id since the last read (see include/ngfreg.h)."""
        ms, cnt = C.c_double(), C.c_int64()
        _check(_lib.load().rg_profile_read(self._ctx, int(kernel), C.byref(ms), C.byref(cnt)), self._ctx,
               "rg_profile_read")
        return ms.value, cnt.value

    def gn_solve(self, u, gn_iters, pcg_iters, ls_max=10, armijo_c=1e-4, drive="host", autotune=False):
        """Runs the fixed Gauss-Newton schedule in place on u; returns (status,
        report) with report rows of RG_REPORT_COLS columns (include/ngfreg.h)."""
        sched = make_schedule(1, gn_iters, pcg_iters, ls_max, armijo_c, drive, autotune)
        rep = np.zeros((gn_iters, RG_REPORT_COLS))
        code = _check(_lib.load().gn_solve(self._ctx, _ptr(self._field(u)), C.byref(sched),
                                           rep.ctypes.data_as(C.POINTER(C.c_double))), self._ctx, "gn_solve")
        return code, rep


def register_pyramid(R, T, h, m_finest, u, params, levels, gn_iters, pcg_iters, ls_max=10, armijo_c=1e-4,
                     kx=None, ky=None, stream=None, drive="host", autotune=False):
    """Multilevel registration; u (finest grid) is updated in place; returns (status, report)."""
    L = _lib.load()
    ig, gg = _img_geom(R.shape, h), _grid_geom(m_finest)
    dtype = _dtype_code(R)
    nk = 0 if kx is None else int(kx.shape[0])
    nbytes = C.c_size_t()
    _check(L.rg_pyramid_workspace_size(C.byref(ig), C.byref(gg), dtype, levels, nk, pcg_iters, C.byref(nbytes)),
           name="rg_pyramid_workspace_size")
    ws = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=R.device)
    wp = (ws.data_ptr() + 255) & ~255
    sched = make_schedule(levels, gn_iters, pcg_iters, ls_max, armijo_c, drive, autotune)
    rep = np.zeros((levels, gn_iters, RG_REPORT_COLS))
    code = L.register_pyramid(C.byref(ig), _ptr(R), _ptr(T), dtype, C.byref(gg), C.byref(params), C.byref(sched), nk,
                              _ptr(kx), _ptr(ky), _ptr(u), rep.ctypes.data_as(C.POINTER(C.c_double)),
                              C.c_void_p(wp), nbytes.value, _stream_ptr(stream))
    if code < 0:
        raise NgfError(code, "register_pyramid")
    return code, rep


def launch_count():
    """Kernels launched by libngfreg.so in this process so far."""
    return int(_lib.load().rg_launch_count())


def restrict_image(img, stream=None):
    n = (C.c_int32 * 3)(img.shape[2], img.shape[1], img.shape[0])
    out = torch.empty((img.shape[0] // 2, img.shape[1] // 2, img.shape[2] // 2), dtype=img.dtype, device=img.device)
    _check(_lib.load().rg_restrict_image(n, _dtype_code(img), _ptr(img), _ptr(out), _stream_ptr(stream)),
           name="rg_restrict_image")
    return out


def prolong_grid(uc, stream=None):
    mc = (C.c_int32 * 3)(uc.shape[3], uc.shape[2], uc.shape[1])
    out = torch.empty((3, 2 * uc.shape[1] - 1, 2 * uc.shape[2] - 1, 2 * uc.shape[3] - 1), dtype=torch.float32,
                      device=uc.device)
    _check(_lib.load().rg_prolong_grid(mc, _ptr(uc), _ptr(out), _stream_ptr(stream)), name="rg_prolong_grid")
    return out
