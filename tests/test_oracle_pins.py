"""Pins for the FP64 oracle: facts the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a closed form, an
invariant, a finite-difference derivative, a brute-force evaluation or a
dense-linear-algebra characterisation that a plausible mistake (dropped term,
wrong sign or index, transposed operand) would break.
"""
import numpy as np
import pytest
from scipy.ndimage import gaussian_filter

import oracle


def smooth_images(n, seed, sigma=1.2, amp=300.0):
    rng = np.random.default_rng(seed)
    shape = (n[2], n[1], n[0])
    R = (amp * gaussian_filter(rng.standard_normal(shape), sigma)).astype(np.float32)
    T = (amp * gaussian_filter(rng.standard_normal(shape), sigma)).astype(np.float32)
    return R, T


def grid_coords(m, g):
    """Node positions [3][mz][my][mx] (mm) of a grid with spacing g."""
    Z, Y, X = np.meshgrid(np.arange(m[2]) * g[2], np.arange(m[1]) * g[1], np.arange(m[0]) * g[0], indexing="ij")
    return np.stack([X, Y, Z])


def voxel_coords(n, h):
    Z, Y, X = np.meshgrid((np.arange(n[2]) + 0.5) * h[2], (np.arange(n[1]) + 0.5) * h[1],
                          (np.arange(n[0]) + 0.5) * h[0], indexing="ij")
    return np.stack([X, Y, Z])


def spacing(n, h, m):
    return tuple(n[a] * h[a] / (m[a] - 1) for a in range(3))


N0, H0, M0 = (16, 16, 8), (1.0, 1.2, 2.5), (5, 5, 3)


@pytest.fixture(scope="module")
def tiny():
    R, T = smooth_images(N0, 1)
    return R, T


# ---------------------------------------------------------------- Eq. (1)
def test_ngf_zero_for_identical_images(tiny):
    R, _ = tiny
    P = oracle.Problem(R, R, H0, M0, eta=10.0, alpha=1.0, gamma=0.1)
    terms, st = P.objective(np.zeros(P.grid_shape))
    assert st == 0
    assert terms[0] == 0.0 and terms[4] == 0.0


def test_ngf_invariant_to_intensity_offset():
    rng = np.random.default_rng(3)
    R = rng.integers(-1000, 100, size=(N0[2], N0[1], N0[0])).astype(np.float32)
    P = oracle.Problem(R, R + np.float32(1024.0), H0, M0, eta=10.0)
    terms, _ = P.objective(np.zeros(P.grid_shape))
    assert terms[0] == 0.0


def test_ngf_closed_form_constant_gradients():
    # R = x-index ramp, T = y-index ramp: f = (1/h1, 0, 0), g = (0, 1/h2, 0) everywhere.
    n, h, m = (8, 8, 8), (0.5, 1.0, 2.0), (5, 5, 5)
    i3, i2, i1 = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    R = i1.astype(np.float32)
    T = i2.astype(np.float32)
    P = oracle.Problem(R, T, h, m, eta=1.0, alpha=0.0)
    terms, _ = P.objective(np.zeros(P.grid_shape))
    # <f,g>_eta = 1, |f|^2_eta = 1 + 4 = 5, |g|^2_eta = 1 + 1 = 2 -> 1 - 1/10 per voxel
    assert terms[0] == pytest.approx(6 ** 3 * 0.9 * (0.5 * 1.0 * 2.0), rel=1e-14)


def test_ngf_pointwise_bounds(tiny):
    R, T = tiny
    P = oracle.Problem(R, T, H0, M0, eta=5.0)
    u = np.random.default_rng(4).normal(0, 0.8, P.grid_shape)
    Tw, _ = P.warp(u)
    D, r, _ = P.ngf_distance(Tw)
    assert np.all(np.abs(r) <= 1.0 + 1e-15)
    nint = np.prod([v - 2 for v in N0])
    assert 0.0 < D < np.prod(H0) * nint


# ------------------------------------------------ trilinear model P and warp
def test_prolong_exact_on_affine_fields():
    n, h, m = (16, 8, 16), (1.0, 2.0, 0.5), (5, 5, 9)
    g = spacing(n, h, m)
    B = np.array([[0.01, -0.02, 0.03], [0.005, 0.0, -0.01], [0.02, 0.01, 0.015]])
    b = np.array([0.3, -0.2, 0.1])
    xn = grid_coords(m, g)
    u = np.einsum("ij,jzyx->izyx", B, xn) + b[:, None, None, None]
    R = np.zeros((n[2], n[1], n[0]), np.float32)
    P = oracle.Problem(R, R, h, m)
    xv = voxel_coords(n, h)
    want = np.einsum("ij,jzyx->izyx", B, xv) + b[:, None, None, None]
    np.testing.assert_allclose(P.prolong(u), want, rtol=0, atol=1e-12)


def test_warp_exact_on_linear_template():
    n, h, m = (16, 16, 8), (1.0, 1.2, 2.5), (5, 5, 3)
    a = np.array([3.0, -2.0, 5.0])
    i3, i2, i1 = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    T = (7.0 + a[0] * i1 + a[1] * i2 + a[2] * i3).astype(np.float32)
    g = spacing(n, h, m)
    B = np.array([[0.02, 0.01, 0.0], [-0.01, 0.03, 0.01], [0.0, 0.02, -0.02]])
    b = np.array([0.7, -0.4, 0.9])
    u = np.einsum("ij,jzyx->izyx", B, grid_coords(m, g)) + b[:, None, None, None]
    P = oracle.Problem(T, T, h, m)
    Tw, dT = P.warp(u)
    xv = voxel_coords(n, h)
    y = xv + np.einsum("ij,jzyx->izyx", B, xv) + b[:, None, None, None]
    s = np.stack([y[k] / h[k] - 0.5 for k in range(3)])
    inside = np.all([(s[k] > 0) & (s[k] < n[k] - 1) for k in range(3)], axis=0)
    want = 7.0 + a[0] * s[0] + a[1] * s[1] + a[2] * s[2]
    assert inside.sum() > 0.5 * inside.size
    np.testing.assert_allclose(Tw[inside], want[inside], rtol=0, atol=1e-9)
    for k in range(3):
        np.testing.assert_allclose(dT[k][inside], a[k] / h[k], rtol=0, atol=1e-9)


def test_warp_integer_voxel_shift_reproduces_voxels(tiny):
    R, T = tiny
    shift = (2, -1, 1)
    P = oracle.Problem(R, T, H0, M0)
    u = np.zeros(P.grid_shape)
    for k in range(3):
        u[k] = shift[k] * H0[k]
    Tw, dT = P.warp(u)
    n = N0
    sl_dst = tuple(slice(max(0, -s), n[k] - max(0, s)) for k, s in reversed(list(enumerate(shift))))
    sl_src = tuple(slice(max(0, s), n[k] - max(0, -s)) for k, s in reversed(list(enumerate(shift))))
    np.testing.assert_allclose(Tw[sl_dst], T[sl_src].astype(np.float64), rtol=0, atol=1e-11)
    # at fraction 0 the derivative is the forward difference T[k+1] - T[k]
    fwd = (T[:, :, 1:].astype(np.float64) - T[:, :, :-1]) / H0[0]
    # voxel (iz, iy, ix) samples T at (iz + 1, iy - 1, ix + 2)
    np.testing.assert_allclose(dT[0][0:n[2] - 1, 1:n[1], 0:n[0] - 3], fwd[1:n[2], 0:n[1] - 1, 2:n[0] - 1],
                               rtol=0, atol=1e-10)


# ----------------------------------------------------- gradient vs FD
def _fd_check(fun, grad, u, rng, eps=1e-5, ndir=6, rel=1e-6):
    for _ in range(ndir):
        d = rng.standard_normal(u.shape)
        d /= np.linalg.norm(d)
        fd = (fun(u + eps * d) - fun(u - eps * d)) / (2 * eps)
        an = float(np.sum(grad * d))
        # truncation O(eps^2) plus FP64 round-off of the objective / eps
        assert abs(fd - an) <= rel * abs(an) + 1e-7 * (np.linalg.norm(grad) + 1.0), (fd, an)


def _kp_problem(R, T, h, m, nk, seed, **kw):
    rng = np.random.default_rng(seed)
    n = (R.shape[2], R.shape[1], R.shape[0])
    fov = np.array(n) * np.array(h)
    kx = rng.uniform(0.05, 0.95, size=(nk, 3)) * fov
    ky = kx + rng.normal(0, 1.0, size=(nk, 3))
    return oracle.Problem(R, T, h, m, kx=kx, ky=ky, **kw)


def test_full_gradient_matches_central_differences(tiny):
    R, T = tiny
    P = _kp_problem(R, T, H0, M0, 40, 5, eta=10.0, alpha=1.0, gamma=0.05, delta=0.3)
    rng = np.random.default_rng(6)
    u = rng.normal(0, 0.5, P.grid_shape)
    terms, g, st = P.gradient(u)
    assert st == 0 and np.all(terms[:4] > 0)
    _fd_check(lambda x: P.objective(x)[0][4], g, u, rng)


@pytest.mark.parametrize("term", ["ngf", "curv", "vcc", "kp"])
def test_term_gradients_match_central_differences(tiny, term):
    R, T = tiny
    P = _kp_problem(R, T, H0, M0, 30, 7, eta=8.0, alpha=1.0, gamma=1.0, delta=1.0)
    rng = np.random.default_rng(8)
    u = rng.normal(0, 0.5, P.grid_shape)
    if term == "ngf":
        f = lambda x: P.ngf_gradient(x)[0]
        g = P.ngf_gradient(u)[1]
    elif term == "curv":
        f = lambda x: P.curvature(x)[0]
        g = P.curvature(u)[1]
    elif term == "vcc":
        f = lambda x: P.vcc(x)[0]
        g = P.vcc(u)[1]
    else:
        f = lambda x: P.keypoints(x)[0]
        g = P.keypoints(u)[1]
    _fd_check(f, g, u, rng)


# ----------------------------------------------------------- Eq. (5)
def test_curvature_zero_for_affine_displacement():
    n, h, m = (16, 16, 8), (1.0, 1.0, 2.0), (9, 9, 5)
    g = spacing(n, h, m)
    # exactly representable affine field
    B = np.array([[0.25, -0.5, 0.125], [0.0625, 0.5, -0.25], [0.125, 0.25, 0.5]])
    u = np.einsum("ij,jzyx->izyx", B, grid_coords(m, g)) + 1.5
    R = np.zeros((n[2], n[1], n[0]), np.float32)
    P = oracle.Problem(R, R, h, m, alpha=1.0)
    e, gr = P.curvature(u)
    assert e == 0.0
    assert np.all(gr == 0.0)


def test_curvature_closed_form_quadratic():
    n, h, m = (16, 16, 8), (1.0, 1.0, 2.0), (9, 5, 5)
    g = spacing(n, h, m)
    u = np.zeros((3, m[2], m[1], m[0]))
    u[0] = (np.arange(m[0]) * g[0])[None, None, :] ** 2     # d2/dx2 = 2 exactly
    R = np.zeros((n[2], n[1], n[0]), np.float32)
    P = oracle.Problem(R, R, h, m)
    e, _ = P.curvature(u)
    ghat = g[0] * g[1] * g[2]
    # L u_x = 2 at the m1-2 x-interior nodes of every (y, z) line, 0 elsewhere
    assert e == pytest.approx(0.5 * ghat * 4.0 * (m[0] - 2) * m[1] * m[2], rel=1e-13)


def test_curvature_hessian_is_linear_symmetric_psd(tiny):
    R, T = tiny
    P = oracle.Problem(R, T, H0, M0)
    rng = np.random.default_rng(9)
    u, v, w = (rng.standard_normal(P.grid_shape) for _ in range(3))
    Hv = P.curvature(u, v)[1]
    diff = P.curvature(u + v)[1] - P.curvature(u)[1]
    np.testing.assert_allclose(Hv, diff, rtol=0, atol=1e-10 * np.abs(Hv).max())
    Hw = P.curvature(u, w)[1]
    assert np.sum(w * Hv) == pytest.approx(np.sum(v * Hw), rel=1e-12)
    assert np.sum(v * Hv) >= 0.0


# ------------------------------------------------------- Eqs. (7)-(9)
def _affine_u(m, g, A):
    return np.einsum("ij,jzyx->izyx", A - np.eye(3), grid_coords(m, g))


def test_vcc_identity():
    R = np.zeros((8, 16, 16), np.float32)
    P = oracle.Problem(R, R, H0, M0, gamma=1.0)
    e, gr, st, (dmin, dmax) = P.vcc(np.zeros(P.grid_shape))
    assert st == 0 and e == 0.0 and dmin == 1.0 and dmax == 1.0
    assert np.all(gr == 0.0)


@pytest.mark.parametrize("s", [2.0, 0.5])
def test_vcc_affine_closed_form_and_symmetry(s):
    n, h, m = (16, 16, 8), (1.0, 1.0, 2.0), (5, 5, 5)
    g = spacing(n, h, m)
    R = np.zeros((n[2], n[1], n[0]), np.float32)
    P = oracle.Problem(R, R, h, m, gamma=1.0)
    A = np.diag([s, 1.0, 1.0])
    e, _, st, (dmin, dmax) = P.vcc(_affine_u(m, g, A))
    assert st == 0 and dmin == pytest.approx(s, rel=1e-14) and dmax == pytest.approx(s, rel=1e-14)
    ncell = (m[0] - 1) * (m[1] - 1) * (m[2] - 1)
    # psi(2) = psi(1/2) = 1/2; 64 bounds per cell, C = cell volume
    assert e == pytest.approx(g[0] * g[1] * g[2] * 64 * ncell * 0.5, rel=1e-13)


def test_vcc_fold_gives_infinity():
    n, h, m = (16, 16, 8), (1.0, 1.0, 2.0), (5, 5, 5)
    g = spacing(n, h, m)
    R = np.zeros((n[2], n[1], n[0]), np.float32)
    P = oracle.Problem(R, R, h, m, gamma=1.0)
    u = _affine_u(m, g, np.diag([-1.0, 1.0, 1.0]))
    e, _, st, _ = P.vcc(u)
    assert st == 1 and np.isinf(e)
    terms, st2 = P.objective(u)
    assert st2 == 1 and np.isinf(terms[4])


def _trilinear_jacobian(u_corners, g, x):
    """Exact grad y at local point x in [0,1]^3 of one cell, y = x + trilinear(u)."""
    J = np.eye(3)
    for o3 in (0, 1):
        for o2 in (0, 1):
            for o1 in (0, 1):
                w = [(x[0] if o1 else 1 - x[0]), (x[1] if o2 else 1 - x[1]), (x[2] if o3 else 1 - x[2])]
                dw = [(1 if o1 else -1) / g[0], (1 if o2 else -1) / g[1], (1 if o3 else -1) / g[2]]
                grad_w = np.array([dw[0] * w[1] * w[2], w[0] * dw[1] * w[2], w[0] * w[1] * dw[2]])
                J += np.outer(u_corners[:, o3, o2, o1], grad_w)
    return J


def test_vcc_brute_force_jacobian_bound():
    """Eq. (8): det grad y(x) = sum_abc lambda_a mu_b nu_c d_abc, hence min d <= det <= max d."""
    n, h, m = (4, 4, 4), (1.0, 1.5, 2.0), (2, 2, 2)
    g = spacing(n, h, m)
    R = np.zeros((4, 4, 4), np.float32)
    P = oracle.Problem(R, R, h, m, gamma=1.0)
    rng = np.random.default_rng(11)
    u = rng.normal(0, 0.25 * min(g), P.grid_shape)
    d = P.vcc_cell_dets(u, (0, 0, 0))       # [a][b][c]
    e, _, st, _ = P.vcc(u)
    assert st == 0
    C = g[0] * g[1] * g[2]
    for _ in range(200):
        x = rng.uniform(0, 1, 3)
        det = np.linalg.det(_trilinear_jacobian(u, g, x))
        # edge index = offset along the lower other axis + 2 * offset along the higher one
        lam = np.array([(1 - x[1]) * (1 - x[2]), x[1] * (1 - x[2]), (1 - x[1]) * x[2], x[1] * x[2]])
        mu = np.array([(1 - x[0]) * (1 - x[2]), x[0] * (1 - x[2]), (1 - x[0]) * x[2], x[0] * x[2]])
        nu = np.array([(1 - x[0]) * (1 - x[1]), x[0] * (1 - x[1]), (1 - x[0]) * x[1], x[0] * x[1]])
        assert np.einsum("a,b,c,abc->", lam, mu, nu, d) == pytest.approx(det, rel=1e-12, abs=1e-13)
        assert d.min() - 1e-12 <= det <= d.max() + 1e-12
        # Eq. (9): V-hat >= C * psi(det) for every point of the cell
        assert e >= C * (det - 1) ** 2 / det


def test_vcc_gn_matrix_is_exact_hessian_where_all_bounds_are_one():
    """psi'(1) = 0, so at a rotation (all d = 1) the GN matrix is the exact Hessian."""
    n, h, m = (16, 16, 8), (1.0, 1.0, 2.0), (5, 5, 5)
    g = spacing(n, h, m)
    R = np.zeros((n[2], n[1], n[0]), np.float32)
    P = oracle.Problem(R, R, h, m, gamma=1.0)
    th = 0.3
    Q = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    u = _affine_u(m, g, Q)
    rng = np.random.default_rng(12)
    v = rng.standard_normal(P.grid_shape)
    eps = 1e-6
    fd = (P.vcc(u + eps * v)[1] - P.vcc(u - eps * v)[1]) / (2 * eps)
    Hv = P.vcc(u, v)[1]
    np.testing.assert_allclose(Hv, fd, rtol=0, atol=1e-6 * np.abs(Hv).max())
    assert np.sum(v * Hv) > 0


# ----------------------------------------------------------- Eq. (10)
def test_keypoints_zero_for_matching_affine_targets(tiny):
    R, T = tiny
    rng = np.random.default_rng(13)
    fov = np.array(N0) * np.array(H0)
    kx = rng.uniform(0.0, 1.0, size=(25, 3)) * fov
    g = spacing(N0, H0, M0)
    B = np.array([[0.01, 0.02, 0.0], [0.0, -0.01, 0.03], [0.02, 0.0, 0.01]])
    b = np.array([1.0, -2.0, 0.5])
    u = np.einsum("ij,jzyx->izyx", B, grid_coords(M0, g)) + b[:, None, None, None]
    ky = kx + kx @ B.T + b
    P = oracle.Problem(R, T, H0, M0, kx=kx, ky=ky, delta=1.0)
    e, gr = P.keypoints(u)
    assert e < 1e-24 and np.abs(gr).max() < 1e-11


def test_keypoint_hessian_exact(tiny):
    R, T = tiny
    P = _kp_problem(R, T, H0, M0, 30, 14, delta=1.0)
    rng = np.random.default_rng(15)
    u, v = rng.standard_normal(P.grid_shape), rng.standard_normal(P.grid_shape)
    Hv = P.keypoints(u, v)[1]
    np.testing.assert_allclose(Hv, P.keypoints(u + v)[1] - P.keypoints(u)[1], rtol=0, atol=1e-10)
    # energy is exactly quadratic: K(u+v) = K(u) + g.v + v.Hv/2
    K0, g0 = P.keypoints(u)
    assert P.keypoints(u + v)[0] == pytest.approx(K0 + np.sum(g0 * v) + 0.5 * np.sum(v * Hv), rel=1e-12)


# ------------------------------------------------ NGF Gauss-Newton matrix
def test_ngf_gn_matrix_against_residual_differences(tiny):
    """H_D = 2 hbar J^T J with J = dr/du: v.H_D w = 2 hbar <Jv, Jw>, J v by central FD of r."""
    R, T = tiny
    P = oracle.Problem(R, T, H0, M0, eta=10.0)
    rng = np.random.default_rng(16)
    u = rng.normal(0, 0.5, P.grid_shape)
    L = P.linearize(u)

    def Jdir(v, eps=1e-5):
        rp = P.ngf_distance(P.warp(u + eps * v)[0])[1]
        rm = P.ngf_distance(P.warp(u - eps * v)[0])[1]
        return (rp - rm) / (2 * eps)

    hb = np.prod(H0)
    v, w = rng.standard_normal(P.grid_shape), rng.standard_normal(P.grid_shape)
    Jv, Jw = Jdir(v), Jdir(w)
    Hv = L.ngf_matvec(v)
    assert np.sum(v * Hv) == pytest.approx(2 * hb * np.sum(Jv * Jv), rel=1e-6)
    assert np.sum(w * Hv) == pytest.approx(2 * hb * np.sum(Jv * Jw), rel=1e-6)
    assert np.sum(w * Hv) == pytest.approx(np.sum(v * L.ngf_matvec(w)), rel=1e-12)


def test_full_gn_matvec_is_sum_of_terms(tiny):
    R, T = tiny
    P = _kp_problem(R, T, H0, M0, 20, 17, eta=10.0, alpha=2.0, gamma=0.1, delta=0.5)
    rng = np.random.default_rng(18)
    u, v = rng.normal(0, 0.3, P.grid_shape), rng.standard_normal(P.grid_shape)
    L = P.linearize(u)
    want = L.ngf_matvec(v) + 2.0 * P.curvature(u, v)[1] + 0.1 * P.vcc(u, v)[1] + 0.5 * P.keypoints(u, v)[1]
    np.testing.assert_allclose(L.matvec(v), want, rtol=1e-12, atol=1e-12 * np.abs(want).max())


# ------------------------------------------------------------- PCG
def _dense(fun, shape):
    nn = int(np.prod(shape))
    H = np.zeros((nn, nn))
    for i in range(nn):
        e = np.zeros(nn)
        e[i] = 1.0
        H[:, i] = fun(e.reshape(shape)).ravel()
    return H


def test_preconditioner_exact_parts_match_dense_assembly():
    """With a constant template (no NGF term) the preconditioner is exactly
    diag(alpha H_R + gamma H_V + delta H_K)."""
    n, h, m = (8, 8, 8), (1.0, 1.0, 2.0), (3, 3, 3)
    R, _ = smooth_images(n, 19)
    T = np.full_like(R, 7.0)
    P = _kp_problem(R, T, h, m, 12, 20, alpha=2.0, gamma=0.3, delta=0.7)
    u = np.random.default_rng(23).normal(0, 0.2, P.grid_shape)
    L = P.linearize(u)
    H = _dense(L.matvec, P.grid_shape)
    np.testing.assert_allclose(L.gn_diag(0.0).ravel(), np.diag(H), rtol=1e-12)
    np.testing.assert_allclose(L.gn_diag(10.0).ravel(), np.diag(H) + 10.0, rtol=1e-12)
    HV = _dense(lambda e: P.vcc(u, e)[1], P.grid_shape)
    np.testing.assert_allclose(P.vcc_diag(u).ravel(), np.diag(HV), rtol=1e-12)


def test_preconditioner_ngf_part_exact_for_isolated_dots():
    """The NGF part drops the cross terms between the six neighbour terms of
    (J e_k)_v; for a template of isolated dots no voxel sees two nonzero terms,
    so it equals the exact diagonal of H_D."""
    n, h, m = (16, 16, 16), (1.0, 1.5, 2.0), (5, 5, 5)
    R, _ = smooth_images(n, 24)
    T = np.zeros_like(R)
    for z in range(3, 14, 5):
        for y in range(3, 14, 5):
            for x in range(3, 14, 5):
                T[z, y, x] = 500.0
    P = oracle.Problem(R, T, h, m, eta=5.0, alpha=0.0)
    L = P.linearize(np.zeros(P.grid_shape))
    H = np.diag(_dense(L.matvec, P.grid_shape))
    d = L.gn_diag(0.0).ravel()
    nz = H > 0
    assert nz.sum() > 100
    np.testing.assert_allclose(d[nz], H[nz], rtol=1e-12)
    assert np.all(d[~nz] == 1.0)          # empty rows fall back to 1


def test_pcg_iterates_minimise_over_krylov_space():
    n, h, m = (8, 8, 8), (1.0, 1.0, 2.0), (3, 3, 3)
    R, T = smooth_images(n, 21)
    P = oracle.Problem(R, T, h, m, eta=5.0, alpha=1.0, gamma=0.01)
    rng = np.random.default_rng(22)
    u = rng.normal(0, 0.3, P.grid_shape)
    L = P.linearize(u)
    H = _dense(L.matvec, P.grid_shape)
    assert np.allclose(H, H.T, rtol=1e-10, atol=1e-10 * np.abs(H).max())
    g = P.gradient(u)[1].ravel()
    Minv = 1.0 / L.gn_diag(0.0).ravel()
    # k-step PCG iterate = argmin of s.Hs/2 + g.s over span{(M^-1 H)^j M^-1 (-g)}
    vecs = [Minv * (-g)]
    for k in range(1, 7):
        Bq, _ = np.linalg.qr(np.stack(vecs, axis=1))
        s_want = Bq @ np.linalg.solve(Bq.T @ H @ Bq, Bq.T @ (-g))
        s_pcg, stats = L.pcg(g.reshape(P.grid_shape), k)
        assert stats[0] == k
        np.testing.assert_allclose(s_pcg.ravel(), s_want, rtol=0, atol=1e-7 * np.abs(s_want).max())
        vecs.append(Minv * (H @ vecs[-1]))
    # long runs converge to the Newton step H s = -g
    s_pcg, _ = L.pcg(g.reshape(P.grid_shape), 400)
    np.testing.assert_allclose(s_pcg.ravel(), np.linalg.solve(H, -g), rtol=0, atol=1e-6 * np.abs(s_pcg).max())


# --------------------------------------------- GN schedule and pyramid
def test_gn_solve_decreases_objective_and_sets_delta():
    from paper_1807_00467_gb300 import phantom
    ph = phantom.make_phantom((32, 32, 16), (2.0, 2.0, 5.0), seed=3, motion="small", n_keypoints=200)
    m = (9, 9, 5)
    P = oracle.Problem(ph.R, ph.T, ph.h, m, eta=10.0, alpha=1.0, gamma=0.001, kx=ph.kp_x, ky=ph.kp_y)
    u0 = np.zeros(P.grid_shape)
    D0 = P.ngf_gradient(u0)[0]
    K0 = P.keypoints(u0)[0]
    u, rep, st = P.gn_solve(u0, gn_iters=3, pcg_iters=10, delta_adaptive=True)
    assert st == 0
    assert P.delta == pytest.approx(D0 / K0, rel=1e-14)          # D = delta K at the start
    assert rep[0, 3] > 0                                          # first step accepted
    for it in range(3):
        if rep[it, 3] > 0:
            assert rep[it, 4] <= rep[it, 1] + 1e-4 * rep[it, 3] * rep[it, 2] + 1e-12
    assert rep[-1, 4] < rep[0, 1]


def test_restriction_and_grid_prolongation_exact_on_linear_data():
    n = (8, 8, 4)
    i3, i2, i1 = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    img = (1.0 + 2 * i1 - 3 * i2 + 0.5 * i3).astype(np.float32)
    c = oracle.restrict_image(img)
    j3, j2, j1 = np.meshgrid(np.arange(2), np.arange(4), np.arange(4), indexing="ij")
    # coarse voxel j has centre at fine index 2j + 1/2
    np.testing.assert_array_equal(c, (1.0 + 2 * (2 * j1 + 0.5) - 3 * (2 * j2 + 0.5) + 0.5 * (2 * j3 + 0.5)).astype(np.float32))
    mc, mf = (3, 3, 2), (5, 5, 3)
    B = np.array([[0.5, 1.0, -2.0], [0.25, 0.0, 1.0], [1.0, -1.0, 0.5]])
    uc = np.einsum("ij,jzyx->izyx", B, grid_coords(mc, (2.0, 2.0, 2.0)))
    uf = oracle.prolong_grid(uc, mf)
    np.testing.assert_allclose(uf, np.einsum("ij,jzyx->izyx", B, grid_coords(mf, (1.0, 1.0, 1.0))), atol=1e-14)


def test_pyramid_reduces_objective():
    from paper_1807_00467_gb300 import phantom
    ph = phantom.make_phantom((32, 32, 16), (2.0, 2.0, 5.0), seed=4, motion="small")
    m = (9, 9, 5)
    P = oracle.Problem(ph.R, ph.T, ph.h, m, eta=10.0, alpha=1.0, gamma=0.001)
    u0 = np.zeros(P.grid_shape)
    J0 = P.objective(u0)[0][4]
    u, rep, st = P.register_pyramid(u0, levels=2, gn_iters=3, pcg_iters=8)
    assert st == 0
    assert P.objective(u)[0][4] < J0


# --------------------------------------------- multilevel driver (Sec. II-D3)
def _pyramid_problem(seed, n_keypoints=0):
    from paper_1807_00467_gb300 import phantom
    ph = phantom.make_phantom((64, 32, 32), (1.5, 2.0, 4.0), seed=seed, motion="small", n_vessels=10,
                              n_keypoints=n_keypoints)
    return ph, (17, 9, 9)


def test_pyramid_with_one_level_is_the_gn_schedule():
    ph, m = _pyramid_problem(30)
    u0 = np.random.default_rng(31).normal(0, 0.5, (3,) + m[::-1])
    P1 = oracle.Problem(ph.R, ph.T, ph.h, m, eta=10.0, alpha=1.0, gamma=0.001)
    u1, rep1, st1 = P1.register_pyramid(u0, levels=1, gn_iters=3, pcg_iters=8)
    P2 = oracle.Problem(ph.R, ph.T, ph.h, m, eta=10.0, alpha=1.0, gamma=0.001)
    u2, rep2, st2 = P2.gn_solve(u0, gn_iters=3, pcg_iters=8)
    assert st1 == st2 == 0
    np.testing.assert_array_equal(u1, u2)
    np.testing.assert_array_equal(rep1[0], rep2)


@pytest.mark.parametrize("levels,kp", [(2, False), (3, True)])
def test_pyramid_is_coarse_solves_and_grid_prolongations(levels, kp):
    """The multilevel driver, decomposed by hand: level l has the images
    restricted l times (2x2x2 box), spacing 2^l h and nodes (m - 1) / 2^l + 1
    per axis; the coarsest start is u0 injected (coarse node k <- fine node
    2^L k); each level runs the Gauss-Newton schedule from the dyadic
    prolongation of the coarser result; delta = D / K is set once, at the
    coarsest start, and carried to the finer levels.  The driver's report rows
    and result must be those of this composition bit for bit, the first row of
    each level must hold J of its own problem at its start, and a wrong
    spacing, grid size, injection node, delta carry or level order breaks it."""
    ph, m = _pyramid_problem(32, n_keypoints=60 if kp else 0)
    kx = ph.kp_x.astype(np.float64) if kp else None
    ky = ph.kp_y.astype(np.float64) if kp else None
    u0 = np.random.default_rng(33).normal(0, 0.5, (3,) + m[::-1])
    kw = dict(eta=10.0, alpha=1.0, gamma=0.001, delta=0.0, kx=kx, ky=ky)
    Pf = oracle.Problem(ph.R, ph.T, ph.h, m, **kw)
    u_pyr, rep_pyr, st = Pf.register_pyramid(u0, levels=levels, gn_iters=2, pcg_iters=6, delta_adaptive=kp)
    assert st == 0
    L = levels - 1
    R, T = [ph.R], [ph.T]
    for _ in range(L):
        R.append(oracle.restrict_image(R[-1]))
        T.append(oracle.restrict_image(T[-1]))
    ml = [tuple((m[a] - 1) // 2 ** l + 1 for a in range(3)) for l in range(levels)]
    hl = [tuple(ph.h[a] * 2 ** l for a in range(3)) for l in range(levels)]
    u = u0[:, ::2 ** L, ::2 ** L, ::2 ** L].copy()
    assert u.shape == (3,) + ml[L][::-1]
    delta = 0.0
    for l in range(L, -1, -1):
        Pl = oracle.Problem(R[l], T[l], hl[l], ml[l], **dict(kw, delta=delta))
        if kp and l == L:
            D0, K0 = Pl.ngf_gradient(u)[0], Pl.keypoints(u)[0]
            delta = D0 / K0
            Pl.delta = delta
        J_start = Pl.objective(u)[0][4]
        u, rep, st_l = Pl.gn_solve(u, gn_iters=2, pcg_iters=6)
        assert st_l == 0
        assert rep[0, 1] == J_start
        np.testing.assert_array_equal(rep, rep_pyr[L - l])
        if l > 0:
            u = oracle.prolong_grid(u, ml[l - 1])
    np.testing.assert_array_equal(u, u_pyr)
    if kp:
        assert Pf.delta == delta and delta > 0.0


# --------------------------------------------- the FP32 cell decision
@pytest.mark.parametrize("name,field", [("tiny", "motion"), ("mid", "motion"), ("mid", "random"), ("full", "motion")])
def test_fp32_cell_decision_is_the_fp64_floor_away_from_knots(name, field):
    """The sample cell is an integer decided in FP32 (the kernels' precision;
    both sides take it the same way).  Against the definition, floor of the
    FP64 sample coordinate s = i + (P u)(x) / h: equal at every voxel farther
    than 1e-4 (voxel units) from an integer, and never more than one cell
    apart; the voxels where the two differ are counted and reported."""
    from paper_1807_00467_gb300 import phantom
    c = phantom.CONFIGS[name]
    ph = phantom.make_phantom(c["n"], c["h"], seed=0, motion=c["motion"])
    m = c["m"]
    u = phantom.motion_on_grid(ph, m, 1.0) if field == "motion" else phantom.random_grid_field(m, 40) * 4.0
    P = oracle.Problem(ph.R, ph.T, ph.h, m)
    k32 = P.cells(u)
    d = P.prolong(u)
    n = P.n
    idx = [np.arange(n[0])[None, None, :], np.arange(n[1])[None, :, None], np.arange(n[2])[:, None, None]]
    differ = 0
    for a in range(3):
        s = idx[a] + d[a] / ph.h[a]
        k64 = np.floor(s)
        far = np.abs(s - np.rint(s)) > 1e-4
        assert np.array_equal(k32[a][far], k64[far].astype(np.int32)), (name, a)
        assert np.abs(k32[a] - k64).max() <= 1
        differ += int((k32[a] != k64).sum())
    print(f"{name} {field}: {differ} of {3 * P.N} cell decisions differ from the FP64 floor (all within 1e-4 of a knot)")
