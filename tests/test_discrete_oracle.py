"""Pins of the discrete-stage oracle (Sec. II-C, Eqs. 2-4) against closed
forms, invariants and brute force on tiny cases."""
import itertools

import numpy as np
import pytest

from oracle import discrete as Dq


def _smooth_noise(shape, seed, sigma=2.0):
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    return (400.0 * gaussian_filter(rng.standard_normal(shape), sigma)).astype(np.float32)


def test_labels_and_mirror():
    d = Dq.label_displacements()
    assert d.shape == (35937, 3)
    assert np.array_equal(d[0], [-32, -32, -32]) and np.array_equal(d[1], [-30, -32, -32])
    assert np.array_equal(d[33], [-32, -30, -32]) and np.array_equal(d[33 * 33], [-32, -32, -30])
    assert np.array_equal(d[17968], [0, 0, 0])
    assert np.array_equal(d[Dq.mirror_labels()], -d)


def test_features_are_unit_eta_vectors():
    img = _smooth_noise((12, 14, 16), 1)
    f = Dq.ngf_features(img, 10.0)
    assert np.allclose(np.linalg.norm(f, axis=-1), 1.0, atol=1e-14)
    # interior gradient: the central difference, x component at (z, y, x) = (5, 6, 7)
    g = 0.5 * (float(img[5, 6, 8]) - float(img[5, 6, 6]))
    assert f[5, 6, 7, 0] * np.sqrt(1.0 / f[5, 6, 7, 3] ** 2) * 10.0 == pytest.approx(g, rel=1e-12)


def test_cost_zero_for_identical_images_at_zero_label():
    img = _smooth_noise((40, 40, 40), 2)
    f = Dq.ngf_features(img, 10.0)
    kps = np.array([[20, 20, 20], [15, 22, 18]])
    D = Dq.cost_volume(f, f, kps, n_steps=5)
    assert np.all(np.abs(D[:, 62]) < 1e-13)          # label 62 = (0, 0, 0) of the 5^3 grid
    assert np.all(D[:, np.arange(125) != 62] > 1e-3)


def test_cost_of_flat_against_ramp_is_closed_form():
    """F constant, M(x) = a . x: r = eta / ||(a, eta)|| for every label, so
    D = |a|^2 / (|a|^2 + eta^2)."""
    n, eta = 30, 10.0
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    a = np.array([3.0, -4.0, 12.0])
    M = (a[0] * x + a[1] * y + a[2] * z).astype(np.float32)
    F = np.full((n, n, n), -850.0, np.float32)
    D = Dq.cost_volume(Dq.ngf_features(F, eta), Dq.ngf_features(M, eta), np.array([[15, 15, 15]]), n_steps=5)
    want = 169.0 / (169.0 + eta * eta)
    assert np.allclose(D, want, rtol=0, atol=1e-13)


def test_shift_is_recovered_by_eq2():
    """M(x) = F(x - s): D(k, s) = 0 exactly, the unique minimum (sign of d)."""
    F = _smooth_noise((48, 48, 48), 3)
    s = (4, -2, 2)                                        # (x, y, z), even
    Mv = np.roll(F, shift=(s[2], s[1], s[0]), axis=(0, 1, 2))
    kps = np.array([[24, 24, 24], [20, 26, 22]])
    D = Dq.cost_volume(Dq.ngf_features(F, 10.0), Dq.ngf_features(Mv, 10.0), kps, n_steps=5)
    d = Dq.label_displacements(5)
    l_s = int(np.flatnonzero((d == s).all(axis=1))[0])
    assert np.all(D[:, l_s] < 1e-13)
    assert np.all(np.argmin(D, axis=1) == l_s)


def test_edge_weights_closed_form():
    kps = np.array([[0, 0, 0], [3, 4, 0], [3, 4, 12]])
    W = Dq.edge_weights(kps, [100.0, -50.0, 100.0])
    assert W.dtype == np.float32
    assert W[0, 1] == np.float32(5.0) + np.float32(150.0) / np.float32(150.0)
    assert W[0, 2] == np.float32(13.0) and W[1, 2] == np.float32(12.0) + np.float32(1.0)
    assert np.all(np.diag(W) == 0) and np.array_equal(W, W.T)


def test_mst_total_matches_scipy_and_is_a_tree():
    from scipy.sparse.csgraph import minimum_spanning_tree
    rng = np.random.default_rng(4)
    kps = rng.integers(0, 60, size=(80, 3))
    kps = np.unique(kps, axis=0)
    W = Dq.edge_weights(kps, rng.normal(-700, 100, size=len(kps)))
    e = Dq.mst(W)
    assert e.shape == (len(kps) - 1, 2)
    ref = minimum_spanning_tree(W.astype(np.float64)).sum()
    assert float(W[e[:, 0], e[:, 1]].astype(np.float64).sum()) == pytest.approx(ref, rel=1e-12)
    order, parent, _ = Dq.tree_order(len(kps), e)
    assert len(order) == len(kps) and (parent >= 0).sum() == len(kps) - 1


def test_mst_brute_force_with_ties():
    """Six vertices with many equal weights: the edge set with the least total
    weight, ties broken by the sorted edge list, over all 6^4 Pruefer trees."""
    W = np.float32([[0, 1, 2, 2, 1, 3], [1, 0, 1, 2, 2, 2], [2, 1, 0, 1, 2, 2],
                    [2, 2, 1, 0, 1, 2], [1, 2, 2, 1, 0, 1], [3, 2, 2, 2, 1, 0]])
    n = 6
    best = None
    for seq in itertools.product(range(n), repeat=n - 2):
        deg = [1] * n
        for v in seq:
            deg[v] += 1
        edges = []
        for v in seq:
            leaf = min(i for i in range(n) if deg[i] == 1)
            edges.append((min(leaf, v), max(leaf, v)))
            deg[leaf] -= 1
            deg[v] -= 1
        a, b = [i for i in range(n) if deg[i] == 1]
        edges.append((a, b))
        # order edges by (w, lo, hi); the MST under a strict order is the
        # lexicographically least sorted weight-key list among the lightest trees
        key = sorted((float(W[x, y]), x, y) for x, y in edges)
        if best is None or key < best:
            best = key
    e = Dq.mst(W)
    assert sorted((float(W[x, y]), x, y) for x, y in e) == best


def test_min_convolve_matches_brute_force():
    rng = np.random.default_rng(5)
    f = rng.random(125)
    d = Dq.label_displacements(5)
    for lam in (0.0, 0.07, 0.5):
        bf = np.array([np.min(f + lam * ((d - d[j]) ** 2).sum(axis=1)) for j in range(125)])
        assert np.allclose(Dq.min_convolve(f, lam, n_steps=5), bf, rtol=0, atol=1e-15)
    assert np.array_equal(Dq.min_convolve(f, np.inf, n_steps=5), f)
    assert np.all(Dq.min_convolve(f, 0.0, n_steps=5) == f.min())


def test_bp_gives_exact_min_marginals():
    """Four keypoints, 27 labels: BP marginals = minimum of the total energy
    over all 27^4 assignments with the keypoint's label fixed."""
    rng = np.random.default_rng(6)
    n, L = 4, 27
    kps = np.array([[0, 0, 0], [3, 0, 0], [3, 5, 0], [0, 1, 7]])
    W = Dq.edge_weights(kps, rng.normal(-700, 200, size=n))
    e = Dq.mst(W)
    D = rng.random((n, L))
    alpha = 0.3
    Mbp = Dq.bp_marginals(D, e, W, alpha, n_steps=3)
    d = Dq.label_displacements(3)
    sq = ((d[:, None, :] - d[None, :, :]) ** 2).sum(axis=2)
    A = np.array(list(itertools.product(range(L), repeat=n)))        # (L^n, n)
    E = D[np.arange(n)[None, :], A].sum(axis=1)
    for a, b in e:
        E = E + alpha / float(W[a, b]) * sq[A[:, a], A[:, b]]
    for k in range(n):
        mk = np.full(L, np.inf)
        np.minimum.at(mk, A[:, k], E)
        assert np.allclose(Mbp[k], mk, rtol=1e-12, atol=1e-12)


def test_symmetric_match_recovers_a_shift():
    """M(x) = F(x - s) with s on the label grid: the forward, backward and
    averaged marginals all pick s (backward picks -s before mirroring)."""
    F = _smooth_noise((96, 96, 96), 7, sigma=2.5)
    s = np.array([6, -4, 10])
    Mv = np.roll(F, shift=(s[2], s[1], s[0]), axis=(0, 1, 2))
    kps = np.array([[48, 48, 48], [44, 52, 50], [52, 46, 44], [47, 50, 53]])
    d1, E1 = Dq.match(F, Mv, kps, symmetric=False)
    d2, E2 = Dq.match(F, Mv, kps, symmetric=True)
    assert np.all(d1 == s) and np.all(d2 == s)


def test_forstner_response_against_direct_inverse():
    """F_D = 1 / trace(S^-1), S by an explicit 3-D convolution with the outer
    product of the Gaussian weights, inverted with numpy."""
    img = _smooth_noise((14, 14, 14), 8, sigma=1.5)
    Rq = Dq.forstner_response(img)
    I = np.pad(img.astype(np.float64), 1, mode="edge")
    g = np.stack([0.5 * (I[1:-1, 1:-1, 2:] - I[1:-1, 1:-1, :-2]), 0.5 * (I[1:-1, 2:, 1:-1] - I[1:-1, :-2, 1:-1]),
                  0.5 * (I[2:, 1:-1, 1:-1] - I[:-2, 1:-1, 1:-1])], axis=-1)
    w = Dq.gaussian_weights()
    K = w[:, None, None] * w[None, :, None] * w[None, None, :]
    r = len(w) // 2
    P = np.pad(g[..., :, None] * g[..., None, :], ((r, r), (r, r), (r, r), (0, 0), (0, 0)), mode="edge")
    for z, y, x in [(7, 7, 7), (5, 9, 6), (8, 4, 10)]:
        S = np.einsum("abc,abcij->ij", K, P[z:z + 2 * r + 1, y:y + 2 * r + 1, x:x + 2 * r + 1])
        assert Rq[z, y, x] == pytest.approx(1.0 / np.trace(np.linalg.inv(S)), rel=1e-10)
    assert Dq.forstner_response(2.0 * img) == pytest.approx(4.0 * Rq, rel=1e-12)   # exact scaling by 2


def test_forstner_zero_for_rank_one_structure():
    z, y, x = np.meshgrid(np.arange(24), np.arange(24), np.arange(24), indexing="ij")
    img = (5.0 * x - 2.0 * y + 3.0 * z).astype(np.float32)      # one gradient direction everywhere
    R = Dq.forstner_response(img)
    assert np.abs(R[8:16, 8:16, 8:16]).max() < 1e-9 * 38.0


def test_forstner_selection_against_brute_force():
    rng = np.random.default_rng(9)
    R = rng.random((9, 10, 11))
    R[2:4, 2:4, 2:4] = 0.0
    mask = rng.random(R.shape) < 0.8
    k = Dq.forstner_select(R, mask)
    want = []
    nz, ny, nx = R.shape
    for zz in range(nz):
        for yy in range(ny):
            for xx in range(nx):
                win = [R[min(max(a, 0), nz - 1), min(max(b, 0), ny - 1), min(max(c, 0), nx - 1)]
                       for a in range(zz - 3, zz + 3) for b in range(yy - 3, yy + 3) for c in range(xx - 3, xx + 3)]
                if mask[zz, yy, xx] and R[zz, yy, xx] > 0 and R[zz, yy, xx] == max(win):
                    want.append((xx, yy, zz))
    assert [tuple(map(int, r)) for r in k] == want


def test_bp_exact_with_a_duplicate_keypoint():
    """A keypoint listed twice: zero edge weight, lambda = inf, so only equal
    labels of the two copies are compatible; brute-force min-marginals over
    all 27^4 labelings with that constraint."""
    rng = np.random.default_rng(11)
    n, L = 4, 27
    kps = np.array([[0, 0, 0], [3, 0, 0], [0, 0, 0], [0, 4, 2]])
    inten = np.array([-700.0, -650.0, -700.0, -820.0], np.float32)
    W = Dq.edge_weights(kps, inten)
    e = Dq.mst(W)
    assert W[0, 2] == 0.0 and [0, 2] in e.tolist()
    D = rng.random((n, L))
    Mbp = Dq.bp_marginals(D, e, W, 0.3, n_steps=3)
    d = Dq.label_displacements(3)
    sq = ((d[:, None, :] - d[None, :, :]) ** 2).sum(axis=2)
    A = np.array(list(itertools.product(range(L), repeat=n)))
    E = D[np.arange(n)[None, :], A].sum(axis=1)
    for a, b in e:
        if W[a, b] == 0.0:
            E = np.where(A[:, a] == A[:, b], E, np.inf)
        else:
            E = E + 0.3 / float(W[a, b]) * sq[A[:, a], A[:, b]]
    for k in range(n):
        mk = np.full(L, np.inf)
        np.minimum.at(mk, A[:, k], E)
        assert np.allclose(Mbp[k], mk, rtol=1e-12, atol=1e-12)
