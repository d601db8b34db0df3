"""The allocation-free NGF distance entry point (ngf_distance_noalloc).

It exists for callers that cannot allocate device memory when they need the
distance (stream capture, host applications that own every device buffer,
fixed memory budgets).  Its result must equal the distance term that the
regular context-based entry point ngf_objective returns, on repeated calls
that reuse the shared static scratch.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from helpers import get_phantom, gpu_context, rel, to_dev

from paper_1807_00467_gb300 import phantom

pytestmark = pytest.mark.gpu

TOL_OBJ = 1e-6


def _geoms(n, h, m):
    from paper_1807_00467_gb300._lib import GridGeom, ImageGeom
    ig, gg = ImageGeom(), GridGeom()
    ig.n[:] = n
    ig.h[:] = h
    gg.m[:] = m
    return ig, gg


def test_noalloc_distance_matches_ngf_objective_twice():
    import torch
    from paper_1807_00467_gb300 import _lib

    L = _lib.load()
    ph = get_phantom("tiny", seed=0)
    m = (17, 17, 13)
    ctx = gpu_context(ph, m, eta=10.0, alpha=1.0, gamma=0.001)
    ig, gg = _geoms(ph.n, ph.h, m)
    D = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for scale in (0.5, 0.8):        # two calls in a row, different displacements
        u = to_dev(phantom.motion_on_grid(ph, m, scale=scale))
        want = ctx.ngf_objective(u)[0].item()
        D.fill_(-1.0)
        code = L.ngf_distance_noalloc(C.byref(ig), C.byref(gg), C.c_void_p(ctx.R.data_ptr()),
                                      C.c_void_p(ctx.T.data_ptr()), C.c_void_p(u.data_ptr()), 10.0,
                                      C.c_void_p(D.data_ptr()), stream)
        torch.cuda.synchronize()
        assert code == 0
        got = D.item()
        print(f"noalloc D = {got:.10e}, ngf_objective D = {want:.10e}")
        assert rel(got, want) <= TOL_OBJ


def test_noalloc_rejects_problems_beyond_the_static_scratch():
    import torch
    from paper_1807_00467_gb300 import _lib

    L = _lib.load()
    # tiles of 28 x 16 voxels in x-y and 32 slices: 74 x 128 x 9 = 85248 > RG_NOALLOC_MAX_CTAS, rejected
    # on the host before any launch
    ig, gg = _geoms((2048, 2048, 288), (0.5, 0.5, 1.0), (513, 513, 145))
    x = torch.zeros(8, device="cuda")
    D = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = C.c_void_p(x.data_ptr())
    code = L.ngf_distance_noalloc(C.byref(ig), C.byref(gg), p, p, p, 10.0, C.c_void_p(D.data_ptr()), None)
    assert code == _lib.RG_ESCRATCH
