"""Several registration problems of uneven sizes in flight on one GPU.

Without keypoints every reduction on the multilevel path has a fixed order,
so each pair registered among others on concurrent streams must give the same
bits as the pair registered alone; the smallest pair is also compared with
the FP64 oracle's multilevel schedule (Sec. II-D3)."""
import numpy as np
import pytest

from paper_1807_00467_gb300 import batch, phantom

from helpers import oracle_problem

TOL_U = 0.01    # mm, final displacement against the oracle


def test_batch_shapes_are_pyramid_ready():
    sh = batch.batch_shapes(n_pairs=200, seed=3)
    v = np.array([np.prod(s) for s in sh], dtype=float)
    for s in sh:
        assert all(e % 16 == 0 for e in s)
        assert 96 <= s[0] <= 512 and 96 <= s[1] <= 512 and 64 <= s[2] <= 128
    # log-uniform counts: roughly half the pairs below the geometric mean
    gm = np.sqrt(96 * 96 * 64 * 512 * 512 * 128.0)
    assert 0.35 < np.mean(v < gm) < 0.65
    assert sh == batch.batch_shapes(n_pairs=200, seed=3)


@pytest.mark.gpu
def test_batch_matches_pairs_one_by_one_and_oracle():
    import torch
    from paper_1807_00467_gb300 import api
    ph = phantom.make_phantom((64, 64, 32), (1.5, 1.5, 3.0), seed=9, motion="small", n_vessels=12, noise_sigma=0.0)
    R, T = torch.from_numpy(ph.R).cuda(), torch.from_numpy(ph.T).cuda()
    shapes = [(64, 64, 32), (48, 56, 32), (56, 48, 24), (40, 40, 16)]
    pairs = batch.crop_pairs(R, T, ph.h, shapes)
    params = api.make_params(eta=10.0, alpha=10.0, gamma=0.001)
    sched = dict(levels=2, gn_iters=2, pcg_iters=10)
    alone = []
    for Rc, Tc, h, m in pairs:
        u = torch.zeros((3,) + m[::-1], device="cuda")
        api.register_pyramid(Rc, Tc, h, m, u, params, **sched)
        alone.append(u)
    us, reps, sec = batch.register_batch(pairs, params, workers=3, **sched)
    for a, b in zip(alone, us):
        assert torch.equal(a, b)
    # the smallest crop against the oracle's multilevel schedule
    Rc, Tc, h, m = pairs[3]
    sub = phantom.Phantom(R=Rc.cpu().numpy(), T=Tc.cpu().numpy(), n=shapes[3], h=ph.h, amps=ph.amps,
                          centres=ph.centres)
    P = oracle_problem(sub, m, alpha=10.0, gamma=0.001)
    uo, repo, st = P.register_pyramid(np.zeros(P.grid_shape), levels=2, gn_iters=2, pcg_iters=10)
    assert st == 0
    np.testing.assert_array_equal(reps[3][..., 3], repo[..., 3])
    d = np.abs(us[3].cpu().numpy() - uo).max()
    print(f"batch: {len(pairs)} pairs in {sec:.3f} s; smallest vs oracle max |du| = {d:.2e} mm")
    assert d <= TOL_U


@pytest.mark.gpu
def test_batched_graph_equals_per_pair_graph_drive():
    """register_pyramid_batch (one graph per level advancing all pairs) gives
    each pair the bits of register_pyramid with the graph drive, FP32 and FP16."""
    import torch
    from paper_1807_00467_gb300 import api
    ph = phantom.make_phantom((64, 64, 32), (1.5, 1.5, 3.0), seed=9, motion="small", n_vessels=12)
    for half in (False, True):
        R, T = torch.from_numpy(ph.R).cuda(), torch.from_numpy(ph.T).cuda()
        if half:
            R, T = (R + 1024.0).half(), (T + 1024.0).half()
        pairs = batch.crop_pairs(R, T, ph.h, [(64, 64, 32), (48, 56, 32), (56, 48, 24), (40, 40, 16)])
        params = api.make_params(eta=10.0, alpha=1.0, gamma=0.001)
        sched = dict(levels=2, gn_iters=3, pcg_iters=10)
        us, reps, sec, code = batch.register_batch_graph(pairs, params, **sched)
        assert code == 0
        for (Rc, Tc, h, m), ub, rb in zip(pairs, us, reps):
            u = torch.zeros((3,) + m[::-1], device="cuda")
            code, rep = api.register_pyramid(Rc, Tc, h, m, u, params, drive="graph", **sched)
            assert code == 0
            np.testing.assert_array_equal(rb, rep)
            assert torch.equal(ub, u)


@pytest.mark.gpu
def test_batched_graph_a_folded_pair_leaves_the_batch():
    """A pair whose start folds (y_x = -x) halts at its first iteration with
    RG_EFOLD: its u keeps the start value and its report stops there; the other
    pairs run to the end with the bits they get on their own."""
    import torch
    from paper_1807_00467_gb300 import _lib, api
    ph = phantom.make_phantom((64, 64, 32), (1.5, 1.5, 3.0), seed=9, motion="small", n_vessels=12)
    R, T = torch.from_numpy(ph.R).cuda(), torch.from_numpy(ph.T).cuda()
    pairs = batch.crop_pairs(R, T, ph.h, [(64, 64, 32), (48, 56, 32), (40, 40, 16)])
    params = api.make_params(eta=10.0, alpha=1.0, gamma=0.001)
    sched = dict(levels=2, gn_iters=2, pcg_iters=8)
    u0 = [torch.zeros((3,) + m[::-1]) for _, _, _, m in pairs]
    m1, h1 = pairs[1][3], pairs[1][2]
    g1 = pairs[1][0].shape[2] * h1[0] / (m1[0] - 1)
    u0[1][0] = -2.0 * torch.arange(m1[0], dtype=torch.float32)[None, None, :] * g1
    us, reps, sec, code = batch.register_batch_graph(pairs, params, u0=u0, **sched)
    assert code == _lib.RG_EFOLD
    assert torch.equal(us[1].cpu(), u0[1])
    assert reps[1][0, 0, 7] == _lib.RG_EFOLD and np.all(reps[1][0, 1:] == 0) and np.all(reps[1][1] == 0)
    for p in (0, 2):
        Rc, Tc, h, m = pairs[p]
        u = torch.zeros((3,) + m[::-1], device="cuda")
        c, rep = api.register_pyramid(Rc, Tc, h, m, u, params, drive="graph", **sched)
        assert c == 0
        np.testing.assert_array_equal(reps[p], rep)
        assert torch.equal(us[p], u)
