"""Tile autotuner: the choice is one of the candidates, is cached per
geometry, and the tuned context still matches the FP64 oracle (objective,
gradient, GN product; the multilevel schedule on a well-conditioned problem)."""
import numpy as np
import pytest

from helpers import gpu_context, oracle_problem, rel, rel_l2, small_phantom, to_dev

from paper_1807_00467_gb300 import phantom

pytestmark = pytest.mark.gpu

TOL_OBJ, TOL_GRAD, TOL_MV, TOL_U = 1e-6, 1e-5, 1e-5, 0.01
CANDIDATES = {(16, 2), (16, 3), (16, 1), (8, 1)}   # column pass, tile pass, general kernels


@pytest.mark.parametrize("shape,h,m", [((64, 64, 48), (1.0, 1.0, 2.5), (17, 17, 13)),
                                       ((96, 80, 32), (1.5, 1.5, 3.0), (25, 21, 9))])
def test_autotuned_context_matches_oracle(shape, h, m):
    ph = small_phantom(shape, h, seed=5)
    u = phantom.motion_on_grid(ph, m, scale=0.5)
    ctx = gpu_context(ph, m, gamma=0.001)
    choice = ctx.autotune(to_dev(u))
    assert choice in CANDIDATES
    assert gpu_context(ph, m, gamma=0.001).autotune(to_dev(u)) == choice   # cached per geometry
    P = oracle_problem(ph, m, gamma=0.001)
    terms, grad = ctx.gn_linearize(to_dev(u))
    ot, og, _ = P.gradient(u)
    assert rel(terms[4].item(), ot[4]) <= TOL_OBJ
    assert rel_l2(grad.cpu().numpy(), og) <= TOL_GRAD
    v = phantom.random_grid_field(m, 7)
    assert rel_l2(ctx.gn_matvec(to_dev(v)).cpu().numpy(), P.linearize(u).matvec(v)) <= TOL_MV
    print(f"{shape}: tile {choice}")


def test_autotuned_pyramid_matches_oracle():
    import torch
    from paper_1807_00467_gb300 import api
    ph = phantom.make_phantom((64, 64, 32), (1.5, 1.5, 3.0), seed=9, motion="small", n_vessels=12, noise_sigma=0.0)
    m = (17, 17, 9)
    R, T = torch.from_numpy(ph.R).cuda(), torch.from_numpy(ph.T).cuda()
    params = api.make_params(eta=10.0, alpha=10.0, gamma=0.001)
    u = torch.zeros((3,) + m[::-1], device="cuda")
    code, rep = api.register_pyramid(R, T, ph.h, m, u, params, levels=2, gn_iters=2, pcg_iters=10, drive="graph",
                                     autotune=True)
    P = oracle_problem(ph, m, alpha=10.0, gamma=0.001)
    uo, repo, st = P.register_pyramid(np.zeros(P.grid_shape), levels=2, gn_iters=2, pcg_iters=10)
    assert code == 0 and st == 0
    np.testing.assert_array_equal(rep[..., 3], repo[..., 3])
    assert np.abs(u.cpu().numpy() - uo).max() <= TOL_U
