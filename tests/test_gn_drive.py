"""The fixed Gauss-Newton schedule (Sec. II-D3) driven three ways: line search
read on the host, decided on the device, and decided on the device with each
iteration replayed from a captured CUDA graph.  The decisions are taken from
the same numbers in the same order, so all three give the same bits: iterate,
report rows and status."""
import numpy as np
import pytest

from helpers import get_phantom, gpu_context, small_phantom

from paper_1807_00467_gb300 import phantom

pytestmark = pytest.mark.gpu

TINY_M = (17, 17, 13)
DRIVES = ("host", "device", "graph")


def _solve_all(ph, m, u0, gn_iters, pcg_iters, ls_max=10, **kw):
    import torch
    out = {}
    for drive in DRIVES:
        ctx = gpu_context(ph, m, **kw)
        u = torch.from_numpy(np.ascontiguousarray(u0, dtype=np.float32)).cuda()
        code, rep = ctx.gn_solve(u, gn_iters=gn_iters, pcg_iters=pcg_iters, ls_max=ls_max, drive=drive)
        torch.cuda.synchronize()
        out[drive] = (code, rep, u.cpu().numpy())
    return out


def _assert_same(out):
    code, rep, u = out["host"]
    for drive in DRIVES[1:]:
        c2, r2, u2 = out[drive]
        assert c2 == code, drive
        np.testing.assert_array_equal(r2, rep, err_msg=drive)
        np.testing.assert_array_equal(u2, u, err_msg=drive)


@pytest.mark.parametrize("gamma", [0.0, 0.001])
def test_drives_agree_tiny(gamma):
    """Also the report's Jacobian bounds (Eqs. (8)-(9)): min d and max d at the
    final iterate against the oracle's 64 bounds per cell at that iterate, and
    the [0.25, 4] flag (with gamma = 0 the objective leaves the volume term out
    and a range pass supplies them)."""
    from helpers import oracle_problem, rel
    ph = get_phantom("tiny", seed=0)
    out = _solve_all(ph, TINY_M, np.zeros((3,) + TINY_M[::-1]), 4, 20, gamma=gamma)
    _assert_same(out)
    rep, u = out["host"][1], out["host"][2]
    assert np.all(rep[:, 3] > 0) and np.all(rep[:, 4] <= rep[:, 1])
    _, _, st, (dmin, dmax) = oracle_problem(ph, TINY_M, gamma=1.0).vcc(u.astype(np.float64))
    print(f"gamma {gamma}: final d range [{rep[-1, 8]:.6f}, {rep[-1, 9]:.6f}] (oracle [{dmin:.6f}, {dmax:.6f}])")
    assert rel(rep[-1, 8], dmin) <= 1e-5 and rel(rep[-1, 9], dmax) <= 1e-5
    assert rep[-1, 10] == float(dmin >= 0.25 and dmax <= 4.0)


def test_drives_agree_with_rejected_steps():
    """Large motion and a one-try line search (ls_max = 0: only t = 1), so
    some steps may be rejected."""
    ph = small_phantom((64, 64, 32), (1.5, 1.5, 3.0), seed=4, motion="large")
    m = (17, 17, 9)
    out = _solve_all(ph, m, np.zeros((3,) + m[::-1]), 5, 15, ls_max=0, gamma=0.001)
    print("accepted t:", out["host"][1][:, 3])
    _assert_same(out)


def test_drives_with_keypoints():
    """With keypoints (their node sums gathered in a fixed order) the drives
    give the same bits too."""
    ph = phantom.make_phantom((64, 64, 32), (1.5, 1.5, 3.0), seed=9, motion="small", n_vessels=12,
                              noise_sigma=0.0, n_keypoints=150)
    m = (17, 17, 9)
    out = _solve_all(ph, m, np.zeros((3,) + m[::-1]), 3, 10, alpha=10.0, gamma=0.001, delta=0.5, kp=True)
    _assert_same(out)


def test_drives_agree_on_a_fold():
    """A folded start: J = +inf, every drive stops with RG_EFOLD at the first
    iteration, u untouched, one report row."""
    from paper_1807_00467_gb300 import api
    ph = get_phantom("tiny", seed=0)
    g = [ph.n[a] * ph.h[a] / (TINY_M[a] - 1) for a in range(3)]
    u0 = np.zeros((3,) + TINY_M[::-1], np.float32)
    u0[0] = -2.0 * (np.arange(TINY_M[0]) * g[0])[None, None, :]
    out = _solve_all(ph, TINY_M, u0, 3, 10, gamma=0.001)
    _assert_same(out)
    code, rep, u = out["graph"]
    assert code == api.RG_EFOLD
    assert np.isinf(rep[0, 1]) and rep[0, 7] == api.RG_EFOLD and np.all(rep[1:] == 0) and np.all(rep[0, 8:] == 0)
    np.testing.assert_array_equal(u, u0)


def test_pyramid_graph_drive_matches_host():
    import torch
    from paper_1807_00467_gb300 import api
    ph = phantom.make_phantom((64, 64, 32), (1.5, 1.5, 3.0), seed=9, motion="small", n_vessels=12, noise_sigma=0.0)
    m = (17, 17, 9)
    R, T = torch.from_numpy(ph.R).cuda(), torch.from_numpy(ph.T).cuda()
    params = api.make_params(eta=10.0, alpha=10.0, gamma=0.001)
    res = {}
    for drive in ("host", "graph"):
        u = torch.zeros((3,) + m[::-1], device="cuda")
        code, rep = api.register_pyramid(R, T, ph.h, m, u, params, levels=2, gn_iters=3, pcg_iters=10, drive=drive)
        res[drive] = (code, rep, u.cpu().numpy())
    assert res["graph"][0] == res["host"][0] == 0
    np.testing.assert_array_equal(res["graph"][1], res["host"][1])
    np.testing.assert_array_equal(res["graph"][2], res["host"][2])


def test_graph_drive_beyond_the_device_report_falls_back_to_host():
    """More iterations than the device keeps report rows for (256): the
    host-driven loop runs instead, with the same bits."""
    import torch
    ph = get_phantom("tiny", seed=0)
    out = {}
    for drive in ("host", "graph"):
        ctx = gpu_context(ph, TINY_M, gamma=0.001)
        u = torch.zeros((3,) + TINY_M[::-1], device="cuda")
        code, rep = ctx.gn_solve(u, gn_iters=260, pcg_iters=2, ls_max=2, drive=drive)
        out[drive] = (code, rep, u.cpu().numpy())
    assert out["host"][0] == out["graph"][0]
    np.testing.assert_array_equal(out["host"][1], out["graph"][1])
    np.testing.assert_array_equal(out["host"][2], out["graph"][2])
