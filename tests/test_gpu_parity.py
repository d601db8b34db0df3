"""GPU path (libngfreg.so through the C ABI) against the FP64 oracle.

Tolerances (stated in the task's numerical targets): objective and its terms
relative error <= 1e-6; gradient and Gauss-Newton products relative L2 error
<= 1e-5; final displacement after a fixed GN-PCG schedule max error <= 0.01 mm.
"""
import numpy as np
import pytest

from helpers import get_phantom, gpu_context, oracle_problem, rel, rel_l2, small_phantom, to_dev

from paper_1807_00467_gb300 import phantom

pytestmark = pytest.mark.gpu

TOL_OBJ, TOL_GRAD, TOL_MV, TOL_U = 1e-6, 1e-5, 1e-5, 0.01

TINY_M = (17, 17, 13)


@pytest.fixture(scope="module")
def tiny():
    return get_phantom("tiny", seed=0)


def _u0(ph, m, scale=0.5):
    return phantom.motion_on_grid(ph, m, scale=scale)


def test_library_loads_on_gpu():
    from paper_1807_00467_gb300 import _lib
    assert b"sm_103a" in _lib.load().rg_version()


@pytest.mark.parametrize("gamma", [0.0, 0.001])
def test_objective_and_gradient_tiny(tiny, gamma):
    u = _u0(tiny, TINY_M)
    ctx = gpu_context(tiny, TINY_M, gamma=gamma)
    terms, grad = ctx.ngf_gradient(to_dev(u))
    terms_o = ctx.ngf_objective(to_dev(u)).cpu().numpy()
    P = oracle_problem(tiny, TINY_M, gamma=gamma)
    ot, og, st = P.gradient(u)
    t = terms.cpu().numpy()
    for k in range(5):
        if ot[k] != 0.0:
            assert rel(t[k], ot[k]) <= TOL_OBJ, (k, t, ot)
    # objective-only pass (line search) sums the same voxels in another order
    np.testing.assert_allclose(terms_o, t, rtol=1e-9)
    err = rel_l2(grad.cpu().numpy(), og)
    print(f"tiny gamma={gamma}: J rel {rel(t[4], ot[4]):.2e}, grad rel-L2 {err:.2e}")
    assert err <= TOL_GRAD


@pytest.mark.parametrize("pass_", [0, 1, 2])
def test_identical_images_give_zero_distance(tiny, pass_):
    """Exactly zero in either objective/gradient pass (0: chosen by size, 1:
    column-marching, 2: tile)."""
    import torch
    from paper_1807_00467_gb300 import _lib, api
    R = torch.from_numpy(tiny.R).cuda()
    ctx = api.Context(R, R.clone(), tiny.h, TINY_M, api.make_params(eta=10.0, alpha=1.0, gamma=0.001))
    ctx.debug_hook(_lib.RG_HOOK_PASS, pass_)
    terms, grad = ctx.ngf_gradient(torch.zeros(ctx.grid_shape, device="cuda"))
    t = terms.cpu().numpy()
    assert t[0] == 0.0 and t[1] == 0.0 and t[2] == 0.0 and t[4] == 0.0
    assert float(grad.abs().max()) == 0.0


def test_gn_matvec_random_vectors_tiny(tiny):
    u = _u0(tiny, TINY_M)
    ctx = gpu_context(tiny, TINY_M, gamma=0.001)
    ctx.gn_linearize(to_dev(u))
    P = oracle_problem(tiny, TINY_M, gamma=0.001)
    L = P.linearize(u)
    for seed in range(100, 110):
        v = phantom.random_grid_field(TINY_M, seed)
        Hv = ctx.gn_matvec(to_dev(v)).cpu().numpy()
        assert rel_l2(Hv, L.matvec(v)) <= TOL_MV, seed


@pytest.mark.parametrize("n,h,m", [((64, 64, 48), (1.0, 1.0, 2.5), (17, 17, 13)),    # rho_z 4
                                   ((96, 48, 36), (0.8, 0.8, 2.5), (25, 13, 19)),    # rho_z 2, chunk tail
                                   ((48, 40, 24), (1.2, 1.2, 2.0), (25, 21, 25)),    # rho_z 1
                                   ((64, 48, 64), (1.0, 1.0, 1.5), (9, 7, 9))])      # rho 8
def test_gn_matvec_dedicated_kernel_matches_general_kernel(n, h, m):
    """Tile height 16 runs the dedicated GN-product kernel, height 8 the general one."""
    ph = small_phantom(n, h, seed=4)
    ctx = gpu_context(ph, m, gamma=0.001)
    ctx.gn_linearize(to_dev(_u0(ph, m, 0.6)))
    v = to_dev(phantom.random_grid_field(m, 21))
    ctx.set_tile(8)
    h8 = ctx.gn_matvec(v).cpu().numpy()
    p8, _ = ctx.gn_pcg_solve(v, 5)          # Jacobi diagonal from the general kernel
    p8 = p8.cpu().numpy()
    ctx.set_tile(16)
    h16 = ctx.gn_matvec(v).cpu().numpy()
    p16, _ = ctx.gn_pcg_solve(v, 5)         # ... and from the dedicated kernel
    assert rel_l2(h16, h8) <= 1e-6
    assert rel_l2(p16.cpu().numpy(), p8) <= 1e-5


@pytest.mark.parametrize("n,h,m,half", [((64, 64, 48), (1.0, 1.0, 2.5), (17, 17, 13), False),
                                        ((96, 48, 36), (0.8, 0.8, 2.5), (25, 13, 19), True),
                                        ((48, 40, 24), (1.2, 1.2, 2.0), (25, 21, 25), False),
                                        ((64, 48, 64), (1.0, 1.0, 1.5), (9, 7, 9), False)])
def test_gradient_pass_matches_general_kernel(n, h, m, half):
    """Tile height 16 runs the persistent objective/gradient pass, height 8 the general kernel."""
    ph = small_phantom(n, h, seed=6)
    ctx = gpu_context(ph, m, gamma=0.001, half=half)
    u = to_dev(_u0(ph, m, 0.6))
    v = to_dev(phantom.random_grid_field(m, 22))
    out = {}
    for ty in (8, 16):
        ctx.set_tile(ty)
        to = ctx.ngf_objective(u).cpu().numpy()
        tg, g = ctx.ngf_gradient(u)
        tl, gl = ctx.gn_linearize(u)
        out[ty] = (to, tg.cpu().numpy(), g.cpu().numpy(), gl.cpu().numpy(), ctx.gn_matvec(v).cpu().numpy())
    for k in range(5):
        if out[8][1][k] != 0.0:
            assert rel(out[16][0][k], out[8][1][k]) <= 1e-6 and rel(out[16][1][k], out[8][1][k]) <= 1e-6, k
    assert rel_l2(out[16][2], out[8][2]) <= 1e-6
    assert rel_l2(out[16][3], out[16][2]) <= 1e-9
    assert rel_l2(out[16][4], out[8][4]) <= 1e-6


@pytest.mark.parametrize("n,h,m,half", [((64, 64, 48), (1.0, 1.0, 2.5), (17, 17, 13), False),
                                        ((96, 48, 36), (0.8, 0.8, 2.5), (25, 13, 19), True),
                                        ((132, 40, 20), (1.0, 1.1, 2.0), (34, 11, 11), False),   # 3 columns, ragged
                                        ((64, 48, 64), (1.0, 1.0, 1.5), (9, 7, 9), False)])      # rho 8
def test_column_pass_matches_tile_pass(n, h, m, half):
    """The column-marching objective / gradient / linearisation pass (forced by
    the test hook at these sizes, where the size rule picks the tile pass)
    against the tile pass: terms, gradient, and the GN product of the stored
    linearisation."""
    from paper_1807_00467_gb300 import _lib
    ph = small_phantom(n, h, seed=8)
    ctx = gpu_context(ph, m, gamma=0.001, half=half)
    u = to_dev(_u0(ph, m, 0.6))
    v = to_dev(phantom.random_grid_field(m, 23))
    out = {}
    for p in (1, 2):
        ctx.debug_hook(_lib.RG_HOOK_PASS, p)
        to = ctx.ngf_objective(u).cpu().numpy()
        tg, g = ctx.ngf_gradient(u)
        tl, gl = ctx.gn_linearize(u)
        out[p] = (to, tg.cpu().numpy(), g.cpu().numpy(), gl.cpu().numpy(), ctx.gn_matvec(v).cpu().numpy())
    ctx.debug_hook(_lib.RG_HOOK_PASS, 0)
    for k in range(5):
        if out[2][1][k] != 0.0:
            assert rel(out[1][0][k], out[2][1][k]) <= 1e-6 and rel(out[1][1][k], out[2][1][k]) <= 1e-6, k
    assert rel_l2(out[1][2], out[2][2]) <= 1e-6
    assert np.array_equal(out[1][3], out[1][2])     # the linearising pass gives the plain gradient's bits
    assert rel_l2(out[1][4], out[2][4]) <= 1e-6


def test_linearize_gradient_matches_plain_gradient(tiny):
    u = to_dev(_u0(tiny, TINY_M))
    ctx = gpu_context(tiny, TINY_M, gamma=0.001)
    t1, g1 = ctx.ngf_gradient(u)
    t2, g2 = ctx.gn_linearize(u)
    assert np.array_equal(t1.cpu().numpy(), t2.cpu().numpy())
    assert np.array_equal(g1.cpu().numpy(), g2.cpu().numpy())


@pytest.mark.parametrize("which", ["curv", "vcc", "kp"])
def test_regularizers(which):
    from paper_1807_00467_gb300 import api
    ph = get_phantom("tiny", seed=1, n_keypoints=300)
    m = TINY_M
    u = _u0(ph, m, 0.8)
    v = phantom.random_grid_field(m, 7)
    ctx = gpu_context(ph, m, gamma=1.0, delta=1.0, kp=True)
    P = oracle_problem(ph, m, gamma=1.0, delta=1.0, kp=True)
    code = {"curv": api.RG_CURV, "vcc": api.RG_VCC, "kp": api.RG_KP}[which]
    fo = {"curv": P.curvature, "vcc": lambda a, b=None: P.vcc(a, b)[:2], "kp": P.keypoints}[which]
    e, g = ctx.regularizer_apply(code, to_dev(u))
    eo, go = fo(u)
    assert rel(e.item(), eo) <= TOL_OBJ
    assert rel_l2(g.cpu().numpy(), go) <= TOL_GRAD
    e2, hv = ctx.regularizer_apply(code, to_dev(u), to_dev(v))
    _, hvo = fo(u, v)
    assert rel_l2(hv.cpu().numpy(), hvo) <= TOL_MV


def test_keypoint_objective_gradient_matvec():
    ph = get_phantom("tiny", seed=2, n_keypoints=500)
    m = TINY_M
    u = _u0(ph, m)
    ctx = gpu_context(ph, m, gamma=0.001, delta=0.3, kp=True)
    P = oracle_problem(ph, m, gamma=0.001, delta=0.3, kp=True)
    terms, grad = ctx.gn_linearize(to_dev(u))
    ot, og, _ = P.gradient(u)
    assert rel(terms[4].item(), ot[4]) <= TOL_OBJ and rel(terms[3].item(), ot[3]) <= TOL_OBJ
    assert rel_l2(grad.cpu().numpy(), og) <= TOL_GRAD
    v = phantom.random_grid_field(m, 101)
    assert rel_l2(ctx.gn_matvec(to_dev(v)).cpu().numpy(), P.linearize(u).matvec(v)) <= TOL_MV


def _crowded_keypoints(ph, m, nk, seed):
    """Keypoints crowded into the 8 cells around one node (many per cell, so
    every node there gathers from several cells), some on nodes, some spread
    over the grid including its faces, two on the far corner (clamped cell,
    fraction 1); targets y = x + N(0, 2 mm)."""
    g = np.array([ph.n[a] * ph.h[a] / (m[a] - 1) for a in range(3)])
    rng = np.random.default_rng(seed)
    node = np.array([m[0] // 2, m[1] // 2, m[2] // 2])
    kx = (node + rng.uniform(-1.0, 1.0, size=(nk, 3))) * g
    kx[: nk // 8] = (node + rng.integers(-1, 2, size=(nk // 8, 3))) * g
    kx[nk // 8: nk // 4] = rng.uniform(0.0, 1.0, size=(nk // 4 - nk // 8, 3)) * g * (np.array(m) - 1)
    kx[-2:] = (np.array(m) - 1) * g
    ky = kx + rng.normal(0.0, 2.0, size=(nk, 3))
    return kx.astype(np.float32), ky.astype(np.float32)


def test_keypoint_node_sums_crowded_cells_are_exact_and_repeatable(tiny):
    """The keypoint penalty (Eq. 10) with many keypoints per cell: energy,
    gradient 2 P^T res and GN product 2 P^T P v against the oracle, the same
    bits on repeated calls (the node sums are gathered in a fixed order), and
    its Jacobi diagonal 2 delta sum w^2 through the first PCG step."""
    import torch

    import oracle
    from paper_1807_00467_gb300 import api
    m = TINY_M
    nk = 400
    kx, ky = _crowded_keypoints(tiny, m, nk, 11)
    u = _u0(tiny, m)
    v = phantom.random_grid_field(m, 12)
    ctx = api.Context(torch.from_numpy(tiny.R).cuda(), torch.from_numpy(tiny.T).cuda(), tiny.h, m,
                      api.make_params(eta=10.0, alpha=1.0, gamma=0.0, delta=5.0), nk_max=nk)
    ctx.set_keypoints(to_dev(kx), to_dev(ky))
    P = oracle.Problem(tiny.R, tiny.T, tiny.h, m, eta=10.0, alpha=1.0, gamma=0.0, delta=5.0,
                       kx=kx.astype(np.float64), ky=ky.astype(np.float64))
    e, gk = ctx.regularizer_apply(api.RG_KP, to_dev(u))
    _, hv = ctx.regularizer_apply(api.RG_KP, to_dev(u), to_dev(v))
    eo, go = P.keypoints(u)
    _, hvo = P.keypoints(u, v)
    assert rel(e.item(), eo) <= TOL_OBJ
    assert rel_l2(gk.cpu().numpy(), go) <= TOL_GRAD
    assert rel_l2(hv.cpu().numpy(), hvo) <= TOL_MV
    for _ in range(3):
        e2, g2 = ctx.regularizer_apply(api.RG_KP, to_dev(u))
        _, h2 = ctx.regularizer_apply(api.RG_KP, to_dev(u), to_dev(v))
        assert e2.item() == e.item() and torch.equal(g2, gk) and torch.equal(h2, hv)
    # the preconditioner: keypoint diagonal dominant at delta = 5
    _, g = ctx.gn_linearize(to_dev(u))
    p, stats = ctx.gn_pcg_solve(g, 1)
    po, so = P.linearize(u).pcg(g.cpu().numpy().astype(np.float64), 1)
    assert stats.cpu().numpy()[0] == so[0] == 1
    assert rel_l2(p.cpu().numpy(), po) <= TOL_GRAD


@pytest.mark.parametrize("n,h,m", [
    ((40, 24, 20), (1.1, 0.9, 2.0), (21, 7, 11)),     # rho (2, 4, 2), ragged tiles in x, y, z
    ((64, 32, 16), (1.0, 1.3, 2.5), (9, 5, 3)),       # rho 8
    ((12, 12, 8), (2.0, 2.0, 3.0), (13, 13, 9)),      # rho 1
    ((96, 48, 36), (0.8, 0.8, 2.5), (25, 13, 19)),    # rho (4, 4, 2), chunk tail
    ((48, 40, 24), (1.2, 1.2, 2.0), (25, 21, 25)),    # rho (2, 2, 1)
])
def test_shapes_and_ratios(n, h, m):
    ph = small_phantom(n, h, seed=5)
    u = _u0(ph, m, 0.7)
    ctx = gpu_context(ph, m, gamma=0.01)
    P = oracle_problem(ph, m, gamma=0.01)
    terms, grad = ctx.gn_linearize(to_dev(u))
    ot, og, _ = P.gradient(u)
    assert rel(terms[4].item(), ot[4]) <= TOL_OBJ
    assert rel_l2(grad.cpu().numpy(), og) <= TOL_GRAD
    v = phantom.random_grid_field(m, 3)
    assert rel_l2(ctx.gn_matvec(to_dev(v)).cpu().numpy(), P.linearize(u).matvec(v)) <= TOL_MV


def test_samples_outside_the_template_are_clamped(tiny):
    u = _u0(tiny, TINY_M)
    u[0, :, :, -3:] += 12.0     # push the samples of a band of voxels past the +x border
    u[2, :2] -= 6.0             # and those of the lowest slices below the first slice
    ctx = gpu_context(tiny, TINY_M)
    P = oracle_problem(tiny, TINY_M)
    terms, grad = ctx.ngf_gradient(to_dev(u))
    ot, og, _ = P.gradient(u)
    Tw, _ = P.warp(u)
    assert rel(terms[4].item(), ot[4]) <= TOL_OBJ
    err = rel_l2(grad.cpu().numpy(), og)
    print(f"clamped band: grad rel-L2 {err:.2e}")
    assert err <= TOL_GRAD


def test_fold_gives_infinite_objective(tiny):
    g = [tiny.n[a] * tiny.h[a] / (TINY_M[a] - 1) for a in range(3)]
    u = np.zeros((3,) + TINY_M[::-1], np.float32)
    u[0] = -2.0 * (np.arange(TINY_M[0]) * g[0])[None, None, :]     # y_x = -x: det < 0
    ctx = gpu_context(tiny, TINY_M, gamma=0.001)
    t = ctx.ngf_objective(to_dev(u)).cpu().numpy()
    assert np.isinf(t[4]) and np.isinf(t[2])


def test_fp16_images_tiny(tiny):
    u = _u0(tiny, TINY_M)
    ctx = gpu_context(tiny, TINY_M, gamma=0.001, half=True)
    P = oracle_problem(tiny, TINY_M, gamma=0.001, half=True)
    terms, grad = ctx.gn_linearize(to_dev(u))
    ot, og, _ = P.gradient(u)
    assert rel(terms[4].item(), ot[4]) <= TOL_OBJ
    assert rel_l2(grad.cpu().numpy(), og) <= TOL_GRAD
    v = phantom.random_grid_field(TINY_M, 104)
    assert rel_l2(ctx.gn_matvec(to_dev(v)).cpu().numpy(), P.linearize(u).matvec(v)) <= TOL_MV


def test_pcg_tiny(tiny):
    u = _u0(tiny, TINY_M)
    ctx = gpu_context(tiny, TINY_M, gamma=0.001)
    terms, g = ctx.gn_linearize(to_dev(u))
    p, stats = ctx.gn_pcg_solve(g, 5)
    P = oracle_problem(tiny, TINY_M, gamma=0.001)
    og = P.gradient(u)[1]
    po, so = P.linearize(u).pcg(og, 5)
    s = stats.cpu().numpy()
    assert s[0] == so[0] == 5
    assert rel_l2(p.cpu().numpy(), po) <= 1e-4


@pytest.mark.parametrize("m,gamma", [(TINY_M, 1.0), ((9, 9, 7), 1.0), (TINY_M, 0.001)])
def test_pcg_first_step_is_the_jacobi_direction(tiny, m, gamma):
    """From p0 = 0 one PCG step is alpha M^-1 g: on the same right-hand side it
    checks the Jacobi diagonal M (NGF, curvature and volume-change parts; the
    volume-change part dominant at gamma = 1, a ragged cell grid in the second
    case) against the oracle's."""
    u = _u0(tiny, m) + phantom.random_grid_field(m, 7, scale=0.2)
    ctx = gpu_context(tiny, m, gamma=gamma)
    _, g = ctx.gn_linearize(to_dev(u))
    p, stats = ctx.gn_pcg_solve(g, 1)
    gh = g.cpu().numpy().astype(np.float64)
    po, so = oracle_problem(tiny, m, gamma=gamma).linearize(u).pcg(gh, 1)
    assert stats.cpu().numpy()[0] == so[0] == 1
    err = rel_l2(p.cpu().numpy(), po)
    print(f"m={m} gamma={gamma}: first PCG step rel-L2 {err:.2e}")
    assert err <= TOL_GRAD


def _replay(ph, m, ctx, u, gn_iters, pcg_iters, steps_checked=None, gamma=0.001):
    """Run the GPU schedule one Gauss-Newton step at a time; the oracle repeats
    chosen steps from the GPU's iterate (per-step parity, 0.01 mm)."""
    P = oracle_problem(ph, m, gamma=gamma)
    worst, reps = 0.0, []
    for k in range(gn_iters):
        uk = u.cpu().numpy().astype(np.float64)
        code, rep = ctx.gn_solve(u, gn_iters=1, pcg_iters=pcg_iters)
        assert code == 0
        reps.append(rep[0])
        if steps_checked is None or k in steps_checked:
            uo, repo, st = P.gn_solve(uk, gn_iters=1, pcg_iters=pcg_iters)
            assert st == 0
            assert rep[0, 3] == repo[0, 3], (k, rep, repo)          # same accepted step length
            assert rel(rep[0, 1], repo[0, 1]) <= TOL_OBJ            # J at the iterate
            d = float(np.abs(u.cpu().numpy() - uo).max())
            worst = max(worst, d)
            assert d <= TOL_U, (k, d)
    return worst, np.array(reps)


def test_gn_solve_tiny(tiny):
    """Five Gauss-Newton steps of 30 PCG steps each: every step within 0.01 mm of
    the oracle's step from the same iterate, the same accepted step lengths, and
    J decreasing monotonically.  On this noisy problem the whole five-step
    trajectory amplifies rounding (the oracle's own endpoint moves ~0.2 mm when
    R changes by one FP32 ulp), so the GPU endpoint is gated against that
    measured sensitivity; the well-conditioned pyramid test gates a whole
    trajectory at 0.01 mm."""
    import torch

    import oracle
    m = TINY_M
    ctx = gpu_context(tiny, m, gamma=0.001)
    u = torch.zeros(ctx.grid_shape, device="cuda")
    worst, rep = _replay(tiny, m, ctx, u, 5, 30)
    print(f"tiny GN replay: worst per-step |du| = {worst:.2e} mm")
    assert np.all(rep[:, 4] <= rep[:, 1])
    P = oracle_problem(tiny, m, gamma=0.001)
    uo, repo, st = P.gn_solve(np.zeros(P.grid_shape), gn_iters=5, pcg_iters=30)
    np.testing.assert_array_equal(rep[:, 3], repo[:, 3])
    # the oracle's own sensitivity: R changed by one ulp (random sign) per voxel
    sens = 0.0
    for seed in (1, 2):
        sgn = np.where(np.random.default_rng(seed).random(tiny.R.shape) < 0.5, -np.inf, np.inf).astype(np.float32)
        Rp = np.nextafter(tiny.R, sgn).astype(np.float32)
        Pp = oracle.Problem(Rp, tiny.T, tiny.h, m, eta=10.0, alpha=1.0, gamma=0.001)
        up, _, _ = Pp.gn_solve(np.zeros(P.grid_shape), gn_iters=5, pcg_iters=30)
        sens = max(sens, float(np.abs(up - uo).max()))
    d = float(np.abs(u.cpu().numpy() - uo).max())
    print(f"tiny GN trajectory: max |u_gpu - u_oracle| = {d:.3e} mm (oracle 1-ulp sensitivity {sens:.3e} mm), "
          f"J {rep[-1, 4]:.6e} vs {repo[-1, 4]:.6e}")
    assert d <= max(TOL_U, 2.0 * sens)
    assert rel(rep[-1, 4], repo[-1, 4]) <= 0.02


def test_pyramid_small():
    """Two levels x 2 GN x 10 PCG on a well-conditioned problem (noise-free
    images, alpha = 10: the oracle's own result moves < 1e-3 mm under 1e-3 HU
    perturbations), so the whole multilevel trajectory can be compared."""
    import torch
    from paper_1807_00467_gb300 import api
    ph = phantom.make_phantom((64, 64, 32), (1.5, 1.5, 3.0), seed=9, motion="small", n_vessels=12, noise_sigma=0.0)
    m = (17, 17, 9)
    R, T = torch.from_numpy(ph.R).cuda(), torch.from_numpy(ph.T).cuda()
    u = torch.zeros((3,) + m[::-1], device="cuda")
    params = api.make_params(eta=10.0, alpha=10.0, gamma=0.001)
    code, rep = api.register_pyramid(R, T, ph.h, m, u, params, levels=2, gn_iters=2, pcg_iters=10)
    P = oracle_problem(ph, m, alpha=10.0, gamma=0.001)
    uo, repo, st = P.register_pyramid(np.zeros(P.grid_shape), levels=2, gn_iters=2, pcg_iters=10)
    assert code == 0 and st == 0
    np.testing.assert_array_equal(rep[..., 3], repo[..., 3])
    d = np.abs(u.cpu().numpy() - uo).max()
    print(f"pyramid: max |du| = {d:.2e} mm")
    assert d <= TOL_U


def test_restrict_and_prolong_grid_against_oracle():
    import torch
    import oracle
    from paper_1807_00467_gb300 import api
    ph = small_phantom((64, 64, 32), (1.5, 1.5, 3.0), seed=9)
    c = api.restrict_image(torch.from_numpy(ph.R).cuda()).cpu().numpy()
    co = oracle.restrict_image(ph.R)
    np.testing.assert_allclose(c, co, rtol=3e-7, atol=0)     # FP32 sum of 8 vs FP64 sum, rounded
    uc = phantom.random_grid_field((9, 9, 5), 3)
    uf = api.prolong_grid(to_dev(uc)).cpu().numpy()
    assert np.abs(uf - oracle.prolong_grid(uc, (17, 17, 9))).max() <= 1e-6


@pytest.mark.slow
def test_mid_config_solve():
    """256x256x64, grid 65x65x33, curvature + VCC, fixed 20 GN x 30 PCG schedule.
    Gate: the oracle repeats steps 0, 5, 10, 15, 19 from the GPU iterate (each
    within 0.01 mm, same line-search step), and the final J agrees within 2 %.
    The final displacements are reported, not gated: at this motion the
    oracle's own 20-step trajectory moves ~3.9 mm under 1e-3 HU of image noise."""
    import torch
    ph = get_phantom("mid", seed=0)
    m = phantom.CONFIGS["mid"]["m"]
    ctx = gpu_context(ph, m, gamma=0.001)
    u = torch.zeros(ctx.grid_shape, device="cuda")
    worst, rep = _replay(ph, m, ctx, u, 20, 30, steps_checked={0, 5, 10, 15, 19})
    P = oracle_problem(ph, m, gamma=0.001)
    uo, repo, st = P.gn_solve(np.zeros(P.grid_shape), gn_iters=20, pcg_iters=30)
    d = np.abs(u.cpu().numpy() - uo).max()
    print(f"mid GN: worst per-step |du| = {worst:.2e} mm, final max |u_gpu - u_oracle| = {d:.3e} mm, "
          f"J {rep[0, 1]:.6e} -> {rep[-1, 4]:.6e} (oracle {repo[-1, 4]:.6e})")
    assert st == 0
    assert rep[-1, 4] < rep[0, 1]
    assert rel(rep[-1, 4], repo[-1, 4]) <= 0.02


def test_full_size_objective_gradient_matvec():
    """512x512x128 (grid 129x129x65) in the launch configuration the benchmark times."""
    ph = get_phantom("full", seed=0)
    m = phantom.CONFIGS["full"]["m"]
    u = _u0(ph, m)
    ctx = gpu_context(ph, m, gamma=0.001)
    terms, grad = ctx.gn_linearize(to_dev(u))
    v = phantom.random_grid_field(m, 105)
    Hv = ctx.gn_matvec(to_dev(v)).cpu().numpy()
    P = oracle_problem(ph, m, gamma=0.001)
    ot, og, _ = P.gradient(u)
    eg, em = rel_l2(grad.cpu().numpy(), og), rel_l2(Hv, P.linearize(u).matvec(v))
    print(f"full size: J rel {rel(terms[4].item(), ot[4]):.2e}, grad rel-L2 {eg:.2e}, Hv rel-L2 {em:.2e}")
    assert rel(terms[4].item(), ot[4]) <= TOL_OBJ
    assert eg <= TOL_GRAD
    assert em <= TOL_MV


def test_entry_points_replay_in_a_cuda_graph(tiny):
    """Objective+gradient, GN product and PCG solve captured on the context's
    stream (outputs preallocated, after one eager call) replay to the same bits."""
    import torch

    from paper_1807_00467_gb300 import api
    s = torch.cuda.Stream()
    R, T = torch.from_numpy(tiny.R).cuda(), torch.from_numpy(tiny.T).cuda()
    ctx = api.Context(R, T, tiny.h, TINY_M, api.make_params(eta=10.0, alpha=1.0, gamma=0.001), stream=s)
    u = to_dev(_u0(tiny, TINY_M))
    v = to_dev(phantom.random_grid_field(TINY_M, 23))
    g, terms, hv, p = (torch.empty_like(u), torch.empty(5, dtype=torch.float64, device="cuda"),
                       torch.empty_like(u), torch.empty_like(u))
    with torch.cuda.stream(s):
        ctx.gn_linearize(u)
        ctx.ngf_gradient(u, g, terms)
        ctx.gn_matvec(v, hv)
        ctx.gn_pcg_solve(v, 10, p)
    s.synchronize()
    eager = [x.clone() for x in (g, terms, hv, p)]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s, capture_error_mode="relaxed"):
        ctx.ngf_gradient(u, g, terms)
        ctx.gn_matvec(v, hv)
        ctx.gn_pcg_solve(v, 10, p)
    for x in (g, terms, hv, p):
        x.zero_()
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        for a, b in zip((g, terms, hv, p), eager):
            assert torch.equal(a, b)


@pytest.mark.parametrize("name,nk", [("tiny", 300), ("mid", 3000)])
def test_adaptive_delta_against_oracle(name, nk):
    """delta = D(u0) / K(u0), set at the start of the schedule (Sec. II-D2):
    the value the GPU keeps (rg_get_params) and the first report row's J equal
    the oracle's at u0 = 0 (the keypoint targets carry the phantom's motion)."""
    import torch

    from paper_1807_00467_gb300 import api
    ph = get_phantom(name, seed=3, n_keypoints=nk)
    m = phantom.CONFIGS[name]["m"]
    dev = torch.device("cuda:0")
    ctx = api.Context(torch.from_numpy(ph.R).to(dev), torch.from_numpy(ph.T).to(dev), ph.h, m,
                      api.make_params(eta=10.0, alpha=1.0, gamma=0.001, delta_adaptive=True), nk_max=nk)
    ctx.set_keypoints(torch.from_numpy(ph.kp_x).to(dev), torch.from_numpy(ph.kp_y).to(dev))
    u = torch.zeros(ctx.grid_shape, device=dev)
    code, rep = ctx.gn_solve(u, gn_iters=1, pcg_iters=5)
    assert code == 0
    delta = ctx.get_params().delta
    P = oracle_problem(ph, m, gamma=0.001, kp=True)
    u0 = np.zeros(P.grid_shape)
    D0, K0 = P.ngf_gradient(u0)[0], P.keypoints(u0)[0]
    P.delta = D0 / K0
    J0 = P.objective(u0)[0][4]
    print(f"{name}, {nk} keypoints: delta {delta:.9e} (oracle {D0 / K0:.9e}), J0 {rep[0, 1]:.9e} (oracle {J0:.9e})")
    assert rel(delta, D0 / K0) <= TOL_OBJ
    assert rel(rep[0, 1], J0) <= TOL_OBJ


def test_fp16_full_size_against_oracle():
    """FP16-stored images (HU + 1024) at 512x512x128 in the benchmark's launch
    configuration, against the oracle run on the FP16-rounded images; the
    quantisation effect itself (oracle on FP32 images vs on FP16-rounded
    images) is reported separately."""
    ph = get_phantom("full", seed=0)
    m = phantom.CONFIGS["full"]["m"]
    u = _u0(ph, m)
    ctx = gpu_context(ph, m, gamma=0.001, half=True)
    terms, grad = ctx.gn_linearize(to_dev(u))
    v = phantom.random_grid_field(m, 106)
    Hv = ctx.gn_matvec(to_dev(v)).cpu().numpy()
    P16 = oracle_problem(ph, m, gamma=0.001, half=True)
    ot, og, _ = P16.gradient(u)
    eJ, eg, em = rel(terms[4].item(), ot[4]), rel_l2(grad.cpu().numpy(), og), rel_l2(Hv, P16.linearize(u).matvec(v))
    P32 = oracle_problem(ph, m, gamma=0.001)
    qt, qg, _ = P32.gradient(u)
    print(f"full size FP16: J rel {eJ:.2e}, grad rel-L2 {eg:.2e}, Hv rel-L2 {em:.2e}; quantisation (oracle FP32 vs "
          f"FP16-rounded images): J rel {rel(ot[4], qt[4]):.2e}, grad rel-L2 {rel_l2(og, qg):.2e}")
    assert eJ <= TOL_OBJ
    assert eg <= TOL_GRAD
    assert em <= TOL_MV
