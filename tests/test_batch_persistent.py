"""The persistent batched PCG (one cooperative kernel running the PCG steps
of every pair of a level, Sec. II-D3's Gauss-Newton solve): the same bits as
the per-pair launches, and its bounded grid barriers.

Each phase of that kernel runs the per-volume kernels' code with the same
partition and reduction order, so every pair must get exactly the iterates
of the batched graph without it (which equals the per-pair graph drive, the
host-driven loop and, within tolerance, the oracle: test_batch.py,
test_gn_drive.py, test_gpu_parity.py)."""
import numpy as np
import pytest

from paper_1807_00467_gb300 import batch, phantom


def _pairs(half):
    import torch
    ph = phantom.make_phantom((160, 112, 48), (1.2, 1.2, 2.5), seed=5, motion="large", n_vessels=16)
    R, T = torch.from_numpy(ph.R).cuda(), torch.from_numpy(ph.T).cuda()
    if half:
        R, T = (R + 1024.0).half(), (T + 1024.0).half()
    # widths from two columns (160) down to below the column kernel's 68 voxels
    # at the coarser level (80 x 64 -> 40 x 32), grids n / 4 + 1; the last pair
    # is never covered and keeps its per-pair launches
    pairs = batch.crop_pairs(R, T, ph.h, [(160, 112, 48), (144, 96, 32), (96, 80, 40), (48, 48, 16)])
    # one pair with rho_z = 2 (grid n_z / 2 + 1)
    Rc, Tc, h, m = pairs[2]
    pairs[2] = (Rc, Tc, h, (m[0], m[1], Rc.shape[0] // 2 + 1))
    return pairs


@pytest.mark.gpu
@pytest.mark.parametrize("half", [False, True])
def test_persistent_batch_equals_batched_graph(half):
    import torch
    from paper_1807_00467_gb300 import api
    pairs = _pairs(half)
    for gamma in (0.001, 0.0):
        params = api.make_params(eta=10.0, alpha=1.0, gamma=gamma)
        sched = dict(levels=2, gn_iters=3, pcg_iters=12)
        ug, rg, _, cg = batch.register_batch_graph(pairs, params, **sched)
        up, rp, _, cp = batch.register_batch_graph(pairs, params, persistent=True, **sched)
        assert cg == cp == 0
        for a, b, ra, rb in zip(ug, up, rg, rp):
            np.testing.assert_array_equal(ra, rb)
            assert torch.equal(a, b)
        # the steps moved the pairs (not a vacuous equality)
        assert all(float(u.abs().max()) > 0.05 for u in up)


@pytest.mark.gpu
def test_persistent_batch_barrier_wait_runs_out():
    """A grid barrier that never completes (the test hook withholds one
    arrival) ends every CTA's bounded wait: the call returns RG_ETIMEOUT, the
    GPU stays usable and the next batch gives the normal result."""
    import torch
    from paper_1807_00467_gb300 import _lib, api
    pairs = _pairs(False)[:2]
    params = api.make_params(eta=10.0, alpha=1.0, gamma=0.001)
    sched = dict(levels=1, gn_iters=1, pcg_iters=4)
    with pytest.raises(api.NgfError) as e:
        batch.register_batch_graph(pairs, params, persistent=True, hook_barrier=True, **sched)
    assert e.value.code == _lib.RG_ETIMEOUT
    ug, rg, _, cg = batch.register_batch_graph(pairs, params, **sched)
    up, rp, _, cp = batch.register_batch_graph(pairs, params, persistent=True, **sched)
    assert cg == cp == 0
    for a, b in zip(ug, up):
        assert torch.equal(a, b)
