"""Many registration problems of uneven sizes on one GPU.

``register_batch`` advances a list of image pairs through the multilevel
Gauss-Newton schedule (``api.register_pyramid`` per pair: restriction, GN-PCG
per level, grid prolongation) with several pairs in flight at once: each
worker owns a CUDA stream and a host thread, pairs are handed out largest
first to the least-loaded worker, so the kernels of small pairs (which leave
most of the GPU idle on their own) overlap with those of other pairs.  The
library calls release the interpreter lock, and every pair's work is ordered
on its worker's stream, so results do not depend on the interleaving.

``batch_shapes`` draws the uneven problem sizes of the batching workload:
voxel counts log-uniform between 96 x 96 x 64 and 512 x 512 x 128, z extent
growing with the cube root of the count, every extent a multiple of 16 (three
pyramid levels over a grid of one node per 4 voxels); ``phantom.batch_pairs``
makes an independent image pair for each.  ``crop_pairs`` instead cuts
centred sub-volumes out of one pair on the device (each a registration
problem of its own under the same motion, at the same spacing).
"""
from __future__ import annotations

import threading
import time

import numpy as np
import torch

from . import api

__all__ = ["batch_shapes", "crop_pairs", "register_batch", "register_batch_graph"]

def batch_shapes(n_pairs=24, seed=0, lo=(96, 96, 64), hi=(512, 512, 128), q=16):
    """[(nx, ny, nz)] of n_pairs problems between the shapes lo and hi."""
    rng = np.random.default_rng(seed)
    v0, v1 = float(np.prod(lo)), float(np.prod(hi))
    rq = lambda x, a, b: int(min(max(int(round(x / q)) * q, a), b))
    out = []
    for _ in range(n_pairs):
        v = np.exp(rng.uniform(np.log(v0), np.log(v1)))
        nz = rq(lo[2] * (v / v0) ** (1.0 / 3.0), lo[2], hi[2] // q * q)
        nx = rq(np.sqrt(v / nz), lo[0], hi[0] // q * q)
        ny = rq(np.sqrt(v / nz), lo[1], hi[1] // q * q)
        out.append((nx, ny, nz))
    return out


def crop_pairs(R, T, h, shapes, grid_step=4):
    """Centred crops [(R_c, T_c, h, m)] of the [nz][ny][nx] device images R, T;
    m = n / grid_step + 1 nodes per axis."""
    out = []
    for n in shapes:
        o = [(R.shape[2 - a] - n[a]) // 2 for a in range(3)]
        sl = (slice(o[2], o[2] + n[2]), slice(o[1], o[1] + n[1]), slice(o[0], o[0] + n[0]))
        m = tuple(n[a] // grid_step + 1 for a in range(3))
        out.append((R[sl].contiguous(), T[sl].contiguous(), tuple(h), m))
    return out


def register_batch_graph(pairs, params, levels, gn_iters, pcg_iters, ls_max=10, armijo_c=1e-4, stream=None, u0=None,
                         persistent=False, hook_barrier=False):
    """All pairs (R, T, h, m) in lockstep through the multilevel schedule with
    one CUDA graph per level advancing every pair's Gauss-Newton iteration
    (register_pyramid_batch); no host threads.  persistent: the PCG steps of
    the pairs whose level the column GN-product kernel covers run in one
    persistent cooperative kernel per iteration (RG_SCHED_PERSISTENT; same
    bits); hook_barrier: test hook, that kernel's grid barriers run out
    (RG_ETIMEOUT).  Returns (displacements, reports, seconds, code): code is
    RG_OK, or the halting status (RG_EFOLD, RG_ENONFINITE) of the
    lowest-numbered pair whose schedule halted; such a pair keeps its start
    value and its report stops at the halting row, the others are complete.
    Other errors raise.  u0: start fields (finest grid) per pair, default
    zero."""
    import ctypes as C

    from . import _lib
    L = _lib.load()
    n = len(pairs)
    dev = pairs[0][0].device
    dtype = api._dtype_code(pairs[0][0])
    igs = (_lib.ImageGeom * n)(*[api._img_geom(R.shape, h) for R, T, h, m in pairs])
    ggs = (_lib.GridGeom * n)(*[api._grid_geom(m) for R, T, h, m in pairs])
    us = [torch.zeros((3, m[2], m[1], m[0]), dtype=torch.float32, device=dev) if u0 is None else
          u0[i].to(device=dev, dtype=torch.float32).contiguous().clone() for i, (R, T, h, m) in enumerate(pairs)]
    wss, wps, wbs = [], [], []
    for i in range(n):
        b = C.c_size_t()
        api._check(L.rg_pyramid_workspace_size(C.byref(igs[i]), C.byref(ggs[i]), dtype, levels, 0, pcg_iters,
                                               C.byref(b)), name="rg_pyramid_workspace_size")
        w = torch.empty(b.value + 256, dtype=torch.uint8, device=dev)
        wss.append(w)
        wps.append((w.data_ptr() + 255) & ~255)
        wbs.append(b.value)
    keep = []

    def ptrs(ts):   # a C array of device pointers, passed as void *
        arr = (C.c_void_p * n)(*[t.data_ptr() for t in ts])
        keep.append(arr)
        return C.cast(arr, C.c_void_p)
    rep = np.zeros((n, levels, gn_iters, _lib.RG_REPORT_COLS))
    sched = api.make_schedule(levels, gn_iters, pcg_iters, ls_max, armijo_c)
    sched.flags = (_lib.RG_SCHED_PERSISTENT if persistent else 0) | (_lib.RG_SCHED_HOOK_BARRIER if hook_barrier else 0)
    wsa = (C.c_void_p * n)(*wps)
    wsp = C.cast(wsa, C.c_void_p)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    code = L.register_pyramid_batch(n, igs, ptrs([p[0] for p in pairs]), ptrs([p[1] for p in pairs]), dtype, ggs,
                                    C.byref(params), C.byref(sched), ptrs(us),
                                    rep.ctypes.data_as(C.POINTER(C.c_double)), wsp, (C.c_size_t * n)(*wbs),
                                    api._stream_ptr(stream))
    torch.cuda.synchronize(dev)
    seconds = time.perf_counter() - t0
    if code < 0 and code != _lib.RG_ENONFINITE:
        raise api.NgfError(code, "register_pyramid_batch")
    return us, list(rep), seconds, code


def register_batch(pairs, params, levels, gn_iters, pcg_iters, workers=4, ls_max=10, armijo_c=1e-4, drive="host",
                   autotune=False):
    """Register every pair (R, T, h, m) (CUDA tensors, float32 or float16 of
    HU + 1024) from u = 0.  Returns (displacements, reports, seconds); the
    displacement of pair i is a float32 tensor (3, m3, m2, m1)."""
    dev = pairs[0][0].device
    order = sorted(range(len(pairs)), key=lambda i: -pairs[i][0].numel())
    load = [0] * workers
    share = [[] for _ in range(workers)]
    for i in order:                       # largest first to the least-loaded worker
        w = min(range(workers), key=lambda k: load[k])
        share[w].append(i)
        load[w] += pairs[i][0].numel()
    us = [None] * len(pairs)
    reps = [None] * len(pairs)
    errors = []

    def run(w):
        try:
            torch.cuda.set_device(dev)
            s = torch.cuda.Stream(device=dev)
            for i in share[w]:
                R, T, h, m = pairs[i]
                with torch.cuda.stream(s):   # u and the workspace belong to this stream
                    u = torch.zeros((3, m[2], m[1], m[0]), dtype=torch.float32, device=dev)
                    code, rep = api.register_pyramid(R, T, h, m, u, params, levels, gn_iters, pcg_iters, ls_max,
                                                     armijo_c, stream=s, drive=drive, autotune=autotune)
                us[i], reps[i] = u, rep
        except Exception as e:   # reported after all workers have stopped
            errors.append(e)

    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    threads = [threading.Thread(target=run, args=(w,)) for w in range(workers) if share[w]]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    torch.cuda.synchronize(dev)
    seconds = time.perf_counter() - t0
    if errors:
        raise errors[0]
    return us, reps, seconds
