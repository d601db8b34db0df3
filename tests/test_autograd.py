"""Differentiation layer (paper_1807_00467_gb300.autograd) on the GPU.

The autograd backward is the library's adjoint kernel.  It is checked against
the FP64 oracle gradient (rel-L2 <= 1e-5) and by central finite differences
of J along random unit grid directions at a 1e-3 mm step.  J is only
piecewise C^1 (trilinear knots), so the finite-difference tolerance is the
oracle's own finite-difference error along the same direction, plus the
propagated objective error of the GPU (|J_gpu - J_oracle| at the two points,
divided by the step).
"""
import numpy as np
import pytest

from helpers import gpu_context, get_phantom, oracle_problem, rel_l2, small_phantom, to_dev

from paper_1807_00467_gb300 import phantom

pytestmark = pytest.mark.gpu

TINY_M = (17, 17, 13)


def _unit_dirs(m, count, seed0=200):
    out = []
    for s in range(seed0, seed0 + count):
        d = phantom.random_grid_field(m, s).astype(np.float64)
        out.append(d / np.linalg.norm(d))
    return out


def _check(ph, m, ndir, eps=1e-3, **kw):
    import torch

    from paper_1807_00467_gb300 import autograd as ag
    ctx = gpu_context(ph, m, **kw)
    P = oracle_problem(ph, m, **kw)
    u = phantom.motion_on_grid(ph, m, scale=0.5).astype(np.float32)
    ut = to_dev(u).requires_grad_(True)
    J = ag.objective(ctx, ut)
    J.backward()
    g = ut.grad.cpu().numpy().astype(np.float64)
    ot, og, _ = P.gradient(u)
    assert abs(J.item() - ot[4]) <= 1e-6 * abs(ot[4])
    assert rel_l2(g, og) <= 1e-5
    gerr = float(np.linalg.norm(g - og))
    # eager form: the same gradient from the fused pass (up to the order of the
    # keypoint adjoint's atomic additions)
    ut2 = to_dev(u).requires_grad_(True)
    ag.objective(ctx, ut2, eager=True).backward()
    assert rel_l2(ut2.grad.cpu().numpy(), ut.grad.cpu().numpy()) <= 1e-6
    worst = 0.0
    rel_fd = []
    for d in _unit_dirs(m, ndir):
        up = (u + eps * d).astype(np.float32)
        um = (u - eps * d).astype(np.float32)
        step = np.float64(up - um)            # the FP32 points actually evaluated
        Jp = ag.objective_terms(ctx, to_dev(up))[4].item()
        Jm = ag.objective_terms(ctx, to_dev(um))[4].item()
        Jpo = P.objective(up)[0][4]
        Jmo = P.objective(um)[0][4]
        fd_gpu, fd_or = Jp - Jm, Jpo - Jmo
        an_gpu, an_or = float((g * step).sum()), float((og * step).sum())
        # fd_gpu - an_gpu = (fd_or - an_or) + (Jp - Jpo) - (Jm - Jmo) - (g - og) . step
        tol = abs(fd_or - an_or) + abs(Jp - Jpo) + abs(Jm - Jmo) + gerr * np.linalg.norm(step) + 1e-12
        err = abs(fd_gpu - an_gpu)
        worst = max(worst, err / tol)
        rel_fd.append((err / max(abs(an_or), 1e-300), abs(fd_or - an_or) / max(abs(an_or), 1e-300)))
        assert err <= tol, (err, tol, fd_gpu, an_gpu, fd_or, an_or)
    r = np.array(rel_fd)
    print(f"relative FD error (median / max): GPU {np.median(r[:, 0]):.2e} / {r[:, 0].max():.2e}, "
          f"oracle {np.median(r[:, 1]):.2e} / {r[:, 1].max():.2e}")
    return worst


def test_autograd_backward_is_the_adjoint_tiny():
    ph = get_phantom("tiny", seed=3, n_keypoints=300)
    w = _check(ph, TINY_M, ndir=8, gamma=0.001, delta=0.3, kp=True)
    print(f"tiny: worst FD error / tolerance {w:.3f}")


def test_autograd_fp16_images_tiny():
    ph = get_phantom("tiny", seed=4)
    _check(ph, TINY_M, ndir=4, gamma=0.001, half=True)


def test_gn_hvp_matches_matvec_and_oracle():
    import torch

    from paper_1807_00467_gb300 import autograd as ag
    ph = get_phantom("tiny", seed=5, n_keypoints=200)
    ctx = gpu_context(ph, TINY_M, gamma=0.001, delta=0.2, kp=True)
    P = oracle_problem(ph, TINY_M, gamma=0.001, delta=0.2, kp=True)
    u = phantom.motion_on_grid(ph, TINY_M, scale=0.5).astype(np.float32)
    v = phantom.random_grid_field(TINY_M, 104)
    hv = ag.gn_hvp(ctx, to_dev(u), to_dev(v)).cpu().numpy()
    assert rel_l2(hv, P.linearize(u).matvec(v)) <= 1e-5
    # symmetric and positive semidefinite in the oracle's FP64 arithmetic
    w = phantom.random_grid_field(TINY_M, 105)
    hw = ag.gn_hvp(ctx, to_dev(u), to_dev(w), relinearize=False).cpu().numpy()
    a, b = float((hv * w).sum()), float((hw * v).sum())
    assert abs(a - b) <= 1e-5 * (abs(a) + abs(b))
    assert float((hv * v).sum()) >= 0.0


@pytest.mark.slow
def test_autograd_mid_with_3000_keypoints_64_directions():
    """256x256x64 (grid 65x65x33), 3000 vessel keypoints with 1 mm noise, adaptive delta."""
    c = phantom.CONFIGS["mid"]
    ph = phantom.make_phantom(c["n"], c["h"], seed=0, motion=c["motion"], n_keypoints=3000)
    m = c["m"]
    import oracle
    P0 = oracle_problem(ph, m, gamma=0.001, kp=True)
    u0 = np.zeros(P0.grid_shape)
    t0, _ = P0.objective(u0)
    delta = t0[0] / t0[3] if t0[3] > 0 else 0.0     # delta = D(u0) / K(u0)
    w = _check(ph, m, ndir=64, gamma=0.001, delta=delta, kp=True)
    print(f"mid: worst FD error / tolerance {w:.3f}")
