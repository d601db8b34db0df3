"""Discrete keypoint stage (Sec. II-C) over torch CUDA tensors: argument
marshalling for the kp_* entry points of libngfreg.so; every step runs in the
library's kernels.

Images: float32 [nz][ny][nx] at 1 mm isotropic spacing.  Keypoints: int32
(nk, 3) voxel positions (x, y, z).  Labels: d = 2 (i - 16) per axis, label
l = (i_z 33 + i_y) 33 + i_x (35 937 labels)."""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from .api import NgfError, _ptr, _stream_ptr

LABELS = 35937


class KpParams(C.Structure):
    _fields_ = [("eta", C.c_double), ("alpha", C.c_double), ("sigma_i", C.c_double)]


def _dims(img):
    return (C.c_int32 * 3)(img.shape[2], img.shape[1], img.shape[0])


def _ok(code, name):
    if code != 0:
        raise NgfError(code, name)


def _scratch(nk, device):
    b = C.c_size_t()
    _ok(_lib.load().kp_scratch_size(int(nk), C.byref(b)), "kp_scratch_size")
    ws = torch.empty(b.value + 256, dtype=torch.uint8, device=device)
    return ws, (ws.data_ptr() + 255) & ~255, b.value


def features(img, eta=10.0, stream=None):
    """(nz, ny, nx, 4) NGF features (grad I, eta) / ||(grad I, eta)||."""
    img = img.contiguous().float()
    out = torch.empty(img.shape + (4,), dtype=torch.float32, device=img.device)
    _ok(_lib.load().kp_ngf_features(_dims(img), _ptr(img), float(eta), _ptr(out), _stream_ptr(stream)),
        "kp_ngf_features")
    return out


def cost_volume(feat_fixed, feat_moving, kps, stream=None):
    """Eq. 2: (nk, 35937) patch costs."""
    kps = kps.contiguous().int()
    D = torch.empty((kps.shape[0], LABELS), dtype=torch.float32, device=kps.device)
    n = (C.c_int32 * 3)(feat_fixed.shape[2], feat_fixed.shape[1], feat_fixed.shape[0])
    _ok(_lib.load().kp_cost_volume(n, _ptr(feat_fixed), _ptr(feat_moving), int(kps.shape[0]), _ptr(kps), _ptr(D),
                                   _stream_ptr(stream)), "kp_cost_volume")
    return D


def mst(kps, intensity, sigma_i=150.0, stream=None):
    """(nk - 1, 2) int32 sorted MST edges (smaller, larger) of Eq. 3's weights."""
    kps = kps.contiguous().int()
    inten = intensity.contiguous().float()
    nk = int(kps.shape[0])
    ws, wp, wb = _scratch(nk, kps.device)
    edges = torch.empty((nk - 1, 2), dtype=torch.int32, device=kps.device)
    _ok(_lib.load().kp_mst(nk, _ptr(kps), _ptr(inten), float(sigma_i), _ptr(edges), C.c_void_p(wp), wb,
                           _stream_ptr(stream)), "kp_mst")
    return edges


def bp_marginals(D, kps, intensity, edges, alpha=0.2, sigma_i=150.0, stream=None):
    """(nk, 35937) exact min-marginals (Eq. 4) on the tree given by edges."""
    kps = kps.contiguous().int()
    inten = intensity.contiguous().float()
    nk = int(kps.shape[0])
    ws, wp, wb = _scratch(nk, kps.device)
    E = torch.empty((nk, LABELS), dtype=torch.float32, device=kps.device)
    _ok(_lib.load().kp_bp_marginals(nk, _ptr(D.contiguous()), _ptr(kps), _ptr(inten), _ptr(edges.contiguous().int()),
                                    float(sigma_i), float(alpha), _ptr(E), C.c_void_p(wp), wb, _stream_ptr(stream)),
        "kp_bp_marginals")
    return E


def forstner(F, mask=None, sigma=1.4, max_kp=100000, response=False, stream=None):
    """Sec. II-C1: (n, 3) int32 keypoints (x, y, z) of the fixed image F
    inside mask (uint8/bool, same shape) in linear index order; with
    response=True also the FP64 distinctiveness F_D."""
    F = F.contiguous().float()
    L = _lib.load()
    b = C.c_size_t()
    _ok(L.kp_forstner_workspace_size(_dims(F), C.byref(b)), "kp_forstner_workspace_size")
    ws = torch.empty(b.value + 256, dtype=torch.uint8, device=F.device)
    wp = (ws.data_ptr() + 255) & ~255
    kps = torch.empty((max_kp, 3), dtype=torch.int32, device=F.device)
    m = None if mask is None else mask.contiguous().to(torch.uint8)
    R = torch.empty(F.shape, dtype=torch.float64, device=F.device) if response else None
    cnt = C.c_int32()
    _ok(L.kp_forstner(_dims(F), _ptr(F), _ptr(m), float(sigma), int(max_kp), _ptr(kps), C.byref(cnt), _ptr(R),
                      C.c_void_p(wp), b.value, _stream_ptr(stream)), "kp_forstner")
    k = kps[: min(cnt.value, max_kp)]
    return (k, R) if response else k


class Matcher:
    """kp_match with a workspace kept for one image shape and keypoint count."""

    def __init__(self, shape, nk, device="cuda", eta=10.0, alpha=0.2, sigma_i=150.0):
        self.n = (C.c_int32 * 3)(shape[2], shape[1], shape[0])
        self.nk = int(nk)
        self.params = KpParams(float(eta), float(alpha), float(sigma_i))
        b = C.c_size_t()
        _ok(_lib.load().kp_workspace_size(self.n, self.nk, C.byref(b)), "kp_workspace_size")
        self._ws = torch.empty(b.value + 256, dtype=torch.uint8, device=device)
        self._wp = (self._ws.data_ptr() + 255) & ~255
        self._wb = b.value
        self.device = device

    def match(self, F, M, kps, symmetric=True, marginals=False, stream=None):
        """Displacements (nk, 3) int32 (voxels = mm) and, if asked, the
        marginals (forward, then backward when symmetric)."""
        kps = kps.contiguous().int()
        disp = torch.empty((self.nk, 3), dtype=torch.int32, device=self.device)
        E = None
        if marginals:
            E = torch.empty(((2 if symmetric else 1) * self.nk, LABELS), dtype=torch.float32, device=self.device)
        _ok(_lib.load().kp_match(self.n, _ptr(F.contiguous()), _ptr(M.contiguous()), self.nk, _ptr(kps),
                                 C.byref(self.params), int(bool(symmetric)), _ptr(disp), _ptr(E), C.c_void_p(self._wp),
                                 self._wb, _stream_ptr(stream)), "kp_match")
        return (disp, E) if marginals else disp


def launch_count():
    return int(_lib.load().kp_launch_count())
