"""Solve results of the configured workloads against the FP64 oracle and the
phantom's known motion u*.

The fixed Gauss-Newton schedule (Sec. II-D3, Eq. (11)) is a non-convex
iteration.  Where the data leave a direction flat (air around the body, far
from any edge), its trajectory amplifies rounding, and no two implementations
can agree to 0.01 mm there.  So the oracle's own sensitivity is measured per
node: the same schedule rerun with R perturbed by Gaussian noise of 1e-3 HU
(two draws; about 1e-6 relative, the size of the FP32 rounding in the GPU's
per-voxel arithmetic).  The GPU result is gated at 0.01 mm against the
oracle on the nodes where that sensitivity is below 0.005 mm.  Reported besides:
max |u_gpu - u_oracle| over all nodes, over nodes whose support lies in the
body and in the lungs, the share of well-conditioned nodes, and the error of
both results against u* on the lung nodes.

The large-motion schedules (mid, the 512x512x128 pyramid, the batch pair)
are chaotic: 1e-3 HU of noise on R moves the oracle's own result by
millimetres at some nodes (mid: at almost every node).  The objective's
derivative jumps where a sample crosses a voxel knot (the trilinear model),
and air voxels with displacements near zero sit on knots, so iterates that
differ in the last bits take different one-sided derivatives there and the
trajectories separate locally, in the oracle as in the GPU path.  There the
GPU result is gated statistically: the percentiles of |u_gpu - u_oracle| over
the nodes may not exceed 1.5 times those of the oracle's own deviation, and
both results must be equally far from u* in the lungs (within 5 %, or within
twice the spread of the perturbed oracle runs); every single step is
checked at 0.01 mm by replaying it in the oracle from the GPU's iterate (here
at the pyramid's finest level, and in test_gpu_parity.py along the tiny and
mid schedules).

Workloads: the tiny configuration (5 GN x 30 PCG), the mid configuration
(20 GN x 30 PCG, volume change), the 512x512x128 3-level pyramid (a shortened
schedule of 2 GN x 10 PCG per level, FP32 images and FP16-stored images), and
the smallest pair of the 24-pair batch (96x96x64, FP16, 3 levels x 10 GN x
30 PCG).  FP16 results are compared with the oracle run on the FP16-rounded
images (every level's restriction rounded to FP16 as the GPU stores it).
"""
import numpy as np
import pytest

from helpers import get_phantom, gpu_context

import oracle
from paper_1807_00467_gb300 import phantom

pytestmark = pytest.mark.gpu

TOL_U, WELL = 0.01, 0.005   # mm: the gate, and the sensitivity below which a node is gated


def _perturbed(R, seed):
    return (R + np.random.default_rng(seed).normal(0.0, 1e-3, R.shape)).astype(np.float32)


def _node_max(d):
    return np.abs(d).max(axis=0)    # over the three components


def _stats(ph, m, u_gpu, u_or, u_moved, label):
    body, lung = phantom.node_regions(ph.n, ph.h, m)
    diff = _node_max(u_gpu - u_or)
    sens = np.max([_node_max(um - u_or) for um in u_moved], axis=0)
    well = sens < WELL
    ustar = phantom.motion_on_grid(ph, m).astype(np.float64)
    selfdev = _node_max(u_moved[0] - u_or)
    st = dict(max_all=float(diff.max()), max_body=float(diff[body].max()), max_lung=float(diff[lung].max()),
              pct_gpu=[float(np.percentile(diff, q)) for q in (50, 90, 99)],
              pct_self=[float(np.percentile(selfdev, q)) for q in (50, 90, 99)],
              max_well=float(diff[well].max()) if well.any() else 0.0, frac_well=float(well.mean()),
              sens_max=float(sens.max()), where_max=("lung" if lung.flat[diff.argmax()] else
                                                     "body" if body.flat[diff.argmax()] else "air"),
              err_true_gpu=float(_node_max(u_gpu - ustar)[lung].mean()),
              err_true_oracle=float(_node_max(u_or - ustar)[lung].mean()),
              err_true_spread=max(abs(float(_node_max(um - ustar)[lung].mean()) - float(_node_max(u_or - ustar)[lung].mean()))
                                  for um in u_moved))
    print(f"{label}: |u_gpu - u_oracle| max {st['max_all']:.3e} (body {st['max_body']:.3e}, lungs "
          f"{st['max_lung']:.3e}, at a {st['where_max']} node); well-conditioned nodes {100 * st['frac_well']:.1f}% "
          f"max {st['max_well']:.3e}; oracle sensitivity max {st['sens_max']:.3e}; mean |u - u*| on lung nodes "
          f"gpu {st['err_true_gpu']:.3f} oracle {st['err_true_oracle']:.3f} mm")
    return st


def _gate(st):
    assert st["frac_well"] > 0.0
    assert st["max_well"] <= TOL_U, st


def _gate_chaotic(st):
    print(f"  percentiles 50/90/99 of |u_gpu - u_oracle| {st['pct_gpu']} mm, of the oracle's own deviation "
          f"{st['pct_self']} mm")
    for a, b in zip(st["pct_gpu"], st["pct_self"]):
        assert a <= max(TOL_U, 1.5 * b), st
    # as far from u* as the oracle (within 5 %, or within 2 times the spread of the perturbed oracle runs)
    assert abs(st["err_true_gpu"] - st["err_true_oracle"]) <= max(0.05 * st["err_true_oracle"],
                                                                  2.0 * st["err_true_spread"]), st


def _oracle_solve(R, T, h, m, gamma, gn, pcg):
    P = oracle.Problem(R, T, h, m, eta=10.0, alpha=1.0, gamma=gamma)
    u, rep, st = P.gn_solve(np.zeros(P.grid_shape), gn_iters=gn, pcg_iters=pcg)
    assert st == 0
    return u


def _half(img):
    return (img + np.float32(1024.0)).astype(np.float16).astype(np.float32)


def _oracle_pyramid(R, T, h, m, levels, gamma, gn, pcg, half):
    """The multilevel schedule (its decomposition, which the oracle pins check
    against orc_register_pyramid bit for bit), with each level's images rounded
    to FP16 when the GPU stores them so."""
    Rs, Ts = [R], [T]
    for _ in range(levels - 1):
        r, t = oracle.restrict_image(Rs[-1]), oracle.restrict_image(Ts[-1])
        if half:   # the restriction of HU + 1024, stored as FP16
            r, t = r.astype(np.float16).astype(np.float32), t.astype(np.float16).astype(np.float32)
        Rs.append(r)
        Ts.append(t)
    L = levels - 1
    u = np.zeros((3,) + tuple((m[a] - 1) // 2 ** L + 1 for a in range(3))[::-1])
    for l in range(L, -1, -1):
        ml = tuple((m[a] - 1) // 2 ** l + 1 for a in range(3))
        hl = tuple(h[a] * 2 ** l for a in range(3))
        P = oracle.Problem(Rs[l], Ts[l], hl, ml, eta=10.0, alpha=1.0, gamma=gamma)
        u, rep, st = P.gn_solve(u, gn_iters=gn, pcg_iters=pcg)
        assert st == 0
        if l > 0:
            u = oracle.prolong_grid(u, tuple((m[a] - 1) // 2 ** (l - 1) + 1 for a in range(3)))
    return u


def _gpu_pyramid(R, T, h, m, levels, gamma, gn, pcg, half):
    import torch

    from paper_1807_00467_gb300 import api
    Rd, Td = torch.from_numpy(R).cuda(), torch.from_numpy(T).cuda()
    if half:
        Rd, Td = (Rd + 1024.0).half(), (Td + 1024.0).half()
    u = torch.zeros((3,) + tuple(m)[::-1], device="cuda")
    code, rep = api.register_pyramid(Rd, Td, h, m, u, api.make_params(eta=10.0, alpha=1.0, gamma=gamma),
                                     levels=levels, gn_iters=gn, pcg_iters=pcg, drive="graph")
    assert code == 0
    return u.cpu().numpy().astype(np.float64)


def test_config1_tiny_solve():
    import torch
    ph = get_phantom("tiny", seed=0)
    m = phantom.CONFIGS["tiny"]["m"]
    ctx = gpu_context(ph, m, gamma=0.0)
    u = torch.zeros(ctx.grid_shape, device="cuda")
    code, rep = ctx.gn_solve(u, gn_iters=5, pcg_iters=30)
    assert code == 0
    uo = _oracle_solve(ph.R, ph.T, ph.h, m, 0.0, 5, 30)
    um = [_oracle_solve(_perturbed(ph.R, s), ph.T, ph.h, m, 0.0, 5, 30) for s in (1, 2)]
    _gate(_stats(ph, m, u.cpu().numpy().astype(np.float64), uo, um, "tiny 5x30"))


@pytest.mark.slow
def test_config2_mid_solve():
    import torch
    ph = get_phantom("mid", seed=0)
    m = phantom.CONFIGS["mid"]["m"]
    ctx = gpu_context(ph, m, gamma=0.001)
    u = torch.zeros(ctx.grid_shape, device="cuda")
    code, rep = ctx.gn_solve(u, gn_iters=20, pcg_iters=30, drive="graph")
    assert code == 0
    uo = _oracle_solve(ph.R, ph.T, ph.h, m, 0.001, 20, 30)
    um = [_oracle_solve(_perturbed(ph.R, s), ph.T, ph.h, m, 0.001, 20, 30) for s in (1, 2)]
    _gate_chaotic(_stats(ph, m, u.cpu().numpy().astype(np.float64), uo, um, "mid 20x30"))


@pytest.mark.slow
@pytest.mark.parametrize("half", [False, True])
def test_config3_full_pyramid_solve(half):
    ph = get_phantom("full", seed=0)
    m = phantom.CONFIGS["full"]["m"]
    R, T = (_half(ph.R), _half(ph.T)) if half else (ph.R, ph.T)
    ug = _gpu_pyramid(ph.R, ph.T, ph.h, m, 3, 0.001, 2, 10, half)
    uo = _oracle_pyramid(R, T, ph.h, m, 3, 0.001, 2, 10, half)
    um = [_oracle_pyramid(_perturbed(R, s), T, ph.h, m, 3, 0.001, 2, 10, half) for s in (1, 2)]
    _gate_chaotic(_stats(ph, m, ug, uo, um, f"512x512x128 3 levels x 2x10 {'FP16' if half else 'FP32'}"))


@pytest.mark.slow
def test_batch_smallest_pair_solve():
    """The smallest pair of the 24-pair batch workload (FP16 images, 3 levels x
    10 GN x 30 PCG), registered by the graph drive (which the batch test shows
    gives each pair the bits of the batched run)."""
    from paper_1807_00467_gb300 import batch
    shapes = batch.batch_shapes()
    k = int(np.argmin([np.prod(s) for s in shapes]))
    n = shapes[k]
    h = tuple(f / n[a] for a, f in enumerate((358.4, 358.4, 320.0)))
    ph = phantom.make_phantom(n, h, seed=k, motion="large")
    m = tuple(n[a] // 4 + 1 for a in range(3))
    ug = _gpu_pyramid(ph.R, ph.T, ph.h, m, 3, 0.001, 10, 30, True)
    R, T = _half(ph.R), _half(ph.T)
    uo = _oracle_pyramid(R, T, ph.h, m, 3, 0.001, 10, 30, True)
    um = [_oracle_pyramid(_perturbed(R, s), T, ph.h, m, 3, 0.001, 10, 30, True) for s in (1, 2)]
    _gate_chaotic(_stats(ph, m, ug, uo, um, f"batch smallest pair {n} FP16 3 levels x 10x30"))


@pytest.mark.slow
def test_config3_finest_level_step_replay():
    """One Gauss-Newton step (10 PCG) at 512x512x128 from the start of the
    pyramid's finest level (the GPU's two coarser levels, prolongated), run on
    the GPU and replayed by the oracle from the same iterate: the same accepted
    step length, J at the iterate within 1e-6, the new iterate within 0.01 mm."""
    import torch

    from paper_1807_00467_gb300 import api
    ph = get_phantom("full", seed=0)
    m = phantom.CONFIGS["full"]["m"]
    R, T = torch.from_numpy(ph.R).cuda(), torch.from_numpy(ph.T).cuda()
    Rh, Th = api.restrict_image(R), api.restrict_image(T)
    mh = tuple((x - 1) // 2 + 1 for x in m)
    uh = torch.zeros((3,) + mh[::-1], device="cuda")
    params = api.make_params(eta=10.0, alpha=1.0, gamma=0.001)
    code, _ = api.register_pyramid(Rh, Th, tuple(2 * x for x in ph.h), mh, uh, params, levels=2, gn_iters=2,
                                   pcg_iters=10, drive="graph")
    assert code == 0
    u0 = api.prolong_grid(uh)
    ctx = gpu_context(ph, m, gamma=0.001)
    u = u0.clone()
    code, rep = ctx.gn_solve(u, gn_iters=1, pcg_iters=10)
    assert code == 0
    P = oracle.Problem(ph.R, ph.T, ph.h, m, eta=10.0, alpha=1.0, gamma=0.001)
    uo, repo, st = P.gn_solve(u0.cpu().numpy().astype(np.float64), gn_iters=1, pcg_iters=10)
    d = float(np.abs(u.cpu().numpy() - uo).max())
    print(f"512x512x128 finest-level step: t {rep[0, 3]} (oracle {repo[0, 3]}), J rel "
          f"{abs(rep[0, 1] - repo[0, 1]) / abs(repo[0, 1]):.2e}, max |du| {d:.3e} mm")
    assert st == 0 and rep[0, 3] == repo[0, 3]
    assert abs(rep[0, 1] - repo[0, 1]) <= 1e-6 * abs(repo[0, 1])
    assert d <= TOL_U
