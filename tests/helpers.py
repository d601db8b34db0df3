"""Shared test helpers: seeded phantoms, GPU contexts and error measures."""
import functools

import numpy as np

from paper_1807_00467_gb300 import phantom


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel(a, b):
    return abs(float(a) - float(b)) / max(abs(float(b)), 1e-300)


@functools.lru_cache(maxsize=8)
def get_phantom(name, seed=0, n_keypoints=0):
    c = phantom.CONFIGS[name]
    return phantom.make_phantom(c["n"], c["h"], seed=seed, motion=c["motion"], n_keypoints=n_keypoints)


@functools.lru_cache(maxsize=8)
def small_phantom(n, h, seed, motion="small", n_keypoints=0):
    return phantom.make_phantom(n, h, seed=seed, motion=motion, n_vessels=12, n_keypoints=n_keypoints)


def gpu_context(ph, m, eta=10.0, alpha=1.0, gamma=0.0, delta=0.0, kp=False, half=False, tau=0.0):
    import torch

    from paper_1807_00467_gb300 import api

    dev = torch.device("cuda:0")
    if half:
        R = torch.from_numpy(ph.R + np.float32(1024.0)).to(dev).half()
        T = torch.from_numpy(ph.T + np.float32(1024.0)).to(dev).half()
    else:
        R = torch.from_numpy(ph.R).to(dev)
        T = torch.from_numpy(ph.T).to(dev)
    nk = len(ph.kp_x) if (kp and ph.kp_x is not None) else 0
    ctx = api.Context(R, T, ph.h, m, api.make_params(eta=eta, alpha=alpha, gamma=gamma, delta=delta, tau=tau),
                      nk_max=nk)
    if nk:
        ctx.set_keypoints(torch.from_numpy(ph.kp_x).to(dev), torch.from_numpy(ph.kp_y).to(dev))
    return ctx


def oracle_problem(ph, m, eta=10.0, alpha=1.0, gamma=0.0, delta=0.0, kp=False, half=False):
    import oracle

    R, T = ph.R, ph.T
    if half:   # the exact values the FP16 path stores, shifted back
        R = (R + np.float32(1024.0)).astype(np.float16).astype(np.float32)
        T = (T + np.float32(1024.0)).astype(np.float16).astype(np.float32)
    kx = ky = None
    if kp and ph.kp_x is not None:
        kx, ky = ph.kp_x.astype(np.float64), ph.kp_y.astype(np.float64)
    return oracle.Problem(R, T, ph.h, m, eta=eta, alpha=alpha, gamma=gamma, delta=delta, kx=kx, ky=ky)


def to_dev(x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to("cuda:0")
