"""FP64 CPU oracle for the discrete keypoint stage of arXiv 1807.00467,
Sec. II-C (Eqs. 2-4 and the symmetric refinement of Sec. II-C4).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg are the only users.  It shares no code with
the GPU library and is never a fallback for it.

Conventions (images at 1 mm isotropic spacing, arrays [z][y][x], positions
(x, y, z) in voxels = mm):

* NGF features: n(x) = (grad I(x), eta) / sqrt(|grad I(x)|^2 + eta^2), the
  central-difference gradient over clamped (edge-replicated) neighbours; then
  <grad M, grad F>_eta / (||grad M||_eta ||grad F||_eta) = n_M . n_F (Eq. 1's
  eta inner product).  A position outside the volume takes the feature of the
  nearest voxel.
* Labels: d = 2 (i - 16) per axis, i = 0..32 (0, +-2, ..., +-32 mm), label
  index l = (i_z 33 + i_y) 33 + i_x; 35 937 labels.
* Patch: the 64 offsets p in {-3, -1, 1, 3}^3 (7^3 voxels at stride 2).
* Eq. 2: D(k, l) = mean_p [1 - (n_M(k + p + d_l) . n_F(k + p))^2].
* Eq. 3: the MST edge weight is w_kq = ||x_k - x_q|| + |F(k) - F(q)| / sigma_I,
  evaluated in FP32 (sqrt, difference, division and sum each rounded once),
  the precision the GPU decides the tree in; edges are ordered by (w, smaller
  index, larger index), a strict total order, so the MST is unique.
* Eq. 4 with the regulariser of Eq. 3, alpha_KP ||d_k - d_q||^2 / w_kq: two
  passes of min-sum belief propagation on the tree rooted at keypoint 0 give
  the exact min-marginals; each message is a min-convolution with a squared
  distance, taken axis by axis (the squared distance is a sum over axes).  A
  zero edge weight (coincident keypoints of the backward search) gives
  lambda = inf: only equal labels are compatible.
* Sec. II-C1 (Foerstner keypoints): S = G_sigma * (grad F grad F^T) with the
  central-difference gradient, a separable Gaussian of sigma = 1.4 voxels
  truncated at radius 5 (weights exp(-i^2 / (2 sigma^2)) normalised to sum 1,
  nearest-voxel extension), F_D = 1 / trace(S^-1) = det S / (sum of the
  principal 2x2 minors) (0 where that sum is 0), F_D* the maximum over the
  6^3 window of offsets -3..2 per axis (nearest-voxel extension); keypoints
  are the voxels of the mask with F_D = F_D* > 0, in linear index order.
* Sec. II-C4: the backward search starts at x_k + d*_k with the images'
  roles swapped (M fixed, F moving, weights from M's intensities); the two
  marginals are averaged with the backward displacement mirrored,
  E(k, d) = (E_fw(k, d) + E_bw(k, -d)) / 2, and d_k = argmin_d E(k, d).
"""
from __future__ import annotations

import numpy as np

N_STEPS = 33                   # labels per axis
LABEL_STEP = 2                 # voxels (mm at 1 mm spacing) between labels
PATCH = (-3, -1, 1, 3)         # patch offsets per axis (7^3 voxels, stride 2)
SIGMA_I = 150.0                # intensity scale of Eq. 3


def label_displacements(n_steps=N_STEPS, step=LABEL_STEP):
    """(L, 3) integer displacements (x, y, z) in label index order."""
    c = step * (np.arange(n_steps) - n_steps // 2)
    dz, dy, dx = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([dx.ravel(), dy.ravel(), dz.ravel()], axis=1)


def mirror_labels(n_steps=N_STEPS):
    """Index of the label -d for every label d."""
    i = np.arange(n_steps ** 3)
    ix, iy, iz = i % n_steps, (i // n_steps) % n_steps, i // (n_steps * n_steps)
    r = n_steps - 1
    return ((r - iz) * n_steps + (r - iy)) * n_steps + (r - ix)


def ngf_features(img, eta):
    """(nz, ny, nx, 4) normalised gradient features (grad I, eta) / ||.||_eta."""
    I = np.pad(np.asarray(img, dtype=np.float64), 1, mode="edge")
    gz = 0.5 * (I[2:, 1:-1, 1:-1] - I[:-2, 1:-1, 1:-1])
    gy = 0.5 * (I[1:-1, 2:, 1:-1] - I[1:-1, :-2, 1:-1])
    gx = 0.5 * (I[1:-1, 1:-1, 2:] - I[1:-1, 1:-1, :-2])
    e = np.full_like(gx, float(eta))
    f = np.stack([gx, gy, gz, e], axis=-1)
    return f / np.sqrt(gx * gx + gy * gy + gz * gz + e * e)[..., None]


def _gather(feat, x, y, z):
    nz, ny, nx = feat.shape[:3]
    return feat[np.clip(z, 0, nz - 1), np.clip(y, 0, ny - 1), np.clip(x, 0, nx - 1)]


def cost_volume(feat_fixed, feat_moving, kps, n_steps=N_STEPS, step=LABEL_STEP):
    """Eq. 2: D[k, l] for keypoints kps (n, 3) integer voxel positions (x, y, z)."""
    kps = np.asarray(kps, dtype=np.int64)
    p = np.array([(px, py, pz) for pz in PATCH for py in PATCH for px in PATCH], dtype=np.int64)   # (64, 3)
    d = label_displacements(n_steps, step)
    D = np.empty((len(kps), len(d)))
    for k, x in enumerate(kps):
        q = x[None, :] + p                                             # (64, 3) patch voxels in F
        nf = _gather(feat_fixed, q[:, 0], q[:, 1], q[:, 2])            # (64, 4)
        s = q[None, :, :] + d[:, None, :]                              # (L, 64, 3) in M
        nm = _gather(feat_moving, s[..., 0], s[..., 1], s[..., 2])     # (L, 64, 4)
        r = np.einsum("lpc,pc->lp", nm, nf)
        D[k] = np.mean(1.0 - r * r, axis=1)
    return D


def edge_weights(kps, intensity, sigma_i=SIGMA_I):
    """(n, n) float32 w_kq of Eq. 3's denominator, each operation rounded to FP32."""
    kps = np.asarray(kps, dtype=np.int64)
    d = kps[:, None, :] - kps[None, :, :]
    dist = np.sqrt((d * d).sum(axis=2).astype(np.float32))
    f = np.asarray(intensity, dtype=np.float32)
    di = np.abs(f[:, None] - f[None, :]) / np.float32(sigma_i)
    return (dist + di).astype(np.float32)


def mst(W):
    """Prim's algorithm from vertex 0 under the order (w, min index, max index).
    Returns the n - 1 edges as (min index, max index) sorted rows."""
    W = np.asarray(W, dtype=np.float32)
    n = W.shape[0]
    if n < 2:
        return np.zeros((0, 2), dtype=np.int64)
    idx = np.arange(n)
    in_tree = np.zeros(n, dtype=bool)
    kw = np.full(n, np.inf, dtype=np.float32)
    klo = np.full(n, n, dtype=np.int64)
    khi = np.full(n, n, dtype=np.int64)
    par = np.full(n, -1, dtype=np.int64)
    edges = []
    u = 0
    for _ in range(n):
        in_tree[u] = True
        if par[u] >= 0:
            edges.append((min(u, par[u]), max(u, par[u])))
        cw, clo, chi = W[u], np.minimum(u, idx), np.maximum(u, idx)
        better = ~in_tree & ((cw < kw) | ((cw == kw) & ((clo < klo) | ((clo == klo) & (chi < khi)))))
        kw[better], klo[better], khi[better], par[better] = cw[better], clo[better], chi[better], u
        cand = np.flatnonzero(~in_tree)
        if len(cand) == 0:
            break
        u = cand[np.lexsort((khi[cand], klo[cand], kw[cand]))[0]]
    e = np.array(edges, dtype=np.int64)
    return e[np.lexsort((e[:, 1], e[:, 0]))]


def tree_order(n, edges, root=0):
    """Breadth-first order from the root, parent of each vertex (-1 at the
    root) and children lists in increasing index order."""
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    parent = np.full(n, -1, dtype=np.int64)
    order, seen = [root], np.zeros(n, dtype=bool)
    seen[root] = True
    i = 0
    while i < len(order):
        k = order[i]
        for q in sorted(adj[k]):
            if not seen[q]:
                seen[q] = True
                parent[q] = k
                order.append(q)
        i += 1
    children = [sorted(q for q in adj[k] if parent[q] == k) for k in range(n)]
    return order, parent, children


def _min_conv_axis(g, C, axis):
    """min over i of g[.., i, ..] + C[i, j] along one axis."""
    g = np.moveaxis(g, axis, -1)
    return np.moveaxis(np.min(g[..., :, None] + C, axis=-2), -1, axis)


def min_convolve(f, lam, n_steps=N_STEPS, step=LABEL_STEP):
    """g(l') = min_l f(l) + lam ||d_l - d_l'||^2 over the label grid, one axis
    at a time; the cost of equal labels is 0 whatever lam (also lam = inf)."""
    i = np.arange(n_steps)
    c = float(step * step) * (i[:, None] - i[None, :]) ** 2            # [from, to]
    C = np.zeros_like(c)
    C[c > 0] = float(lam) * c[c > 0]
    g = np.asarray(f, dtype=np.float64).reshape(n_steps, n_steps, n_steps)   # [z][y][x]
    for axis in (2, 1, 0):                                              # x, then y, then z
        g = _min_conv_axis(g, C, axis)
    return g.ravel()


def bp_marginals(D, edges, W, alpha, n_steps=N_STEPS, step=LABEL_STEP, root=0):
    """Exact min-marginals of sum_k D(k, d_k) + sum_edges alpha ||d_k - d_q||^2 / w_kq
    by two passes of min-sum messages (Eq. 4) on the tree."""
    n = D.shape[0]
    order, parent, children = tree_order(n, edges, root)
    with np.errstate(divide="ignore"):   # a zero weight gives lambda = inf
        lam = {k: float(np.float64(alpha) / np.float64(W[k, parent[k]])) for k in range(n) if parent[k] >= 0}
    up = {}
    for k in reversed(order):
        if parent[k] < 0:
            continue
        h = D[k] + sum((up[c] for c in children[k]), np.zeros(D.shape[1]))
        up[k] = min_convolve(h, lam[k], n_steps, step)
    M = np.empty_like(D, dtype=np.float64)
    for k in order:
        s = D[k] + sum((up[c] for c in children[k]), np.zeros(D.shape[1]))
        if parent[k] >= 0:
            q = parent[k]
            s = s + min_convolve(M[q] - up[k], lam[k], n_steps, step)
        M[k] = s
    return M


def match(F, Mv, kps, eta=10.0, alpha=0.2, sigma_i=SIGMA_I, symmetric=True):
    """Regularised displacements (n, 3) of keypoints kps (voxels) from the
    fixed image F to the moving image Mv (Sec. II-C2-4), with the marginals:
    returns (d, E) where E is the (averaged) marginal energy."""
    kps = np.asarray(kps, dtype=np.int64)
    fF, fM = ngf_features(F, eta), ngf_features(Mv, eta)
    disp = label_displacements()

    def one_way(ffix, fmov, img_fix, pts):
        D = cost_volume(ffix, fmov, pts)
        nz, ny, nx = img_fix.shape
        inten = img_fix[np.clip(pts[:, 2], 0, nz - 1), np.clip(pts[:, 1], 0, ny - 1), np.clip(pts[:, 0], 0, nx - 1)]
        W = edge_weights(pts, inten, sigma_i)
        return bp_marginals(D, mst(W), W, alpha)

    E = one_way(fF, fM, np.asarray(F, np.float32), kps)
    if symmetric:
        d1 = disp[np.argmin(E, axis=1)]
        Eb = one_way(fM, fF, np.asarray(Mv, np.float32), kps + d1)
        E = 0.5 * (E + Eb[:, mirror_labels()])
    return disp[np.argmin(E, axis=1)], E


FORSTNER_SIGMA = 1.4           # mm (= voxels at 1 mm)
FORSTNER_RADIUS = 5            # Gaussian taps -5..5
FORSTNER_BOX = 6               # side of the maximum filter's cube


def gaussian_weights(sigma=FORSTNER_SIGMA, radius=FORSTNER_RADIUS):
    i = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-(i * i) / (2.0 * sigma * sigma))
    return w / w.sum()


def forstner_response(F, sigma=FORSTNER_SIGMA, radius=FORSTNER_RADIUS):
    """F_D = 1 / trace((G_sigma * grad F grad F^T)^-1) per voxel (FP64)."""
    from scipy.ndimage import correlate1d
    I = np.pad(np.asarray(F, dtype=np.float64), 1, mode="edge")
    g = [0.5 * (I[1:-1, 1:-1, 2:] - I[1:-1, 1:-1, :-2]),
         0.5 * (I[1:-1, 2:, 1:-1] - I[1:-1, :-2, 1:-1]),
         0.5 * (I[2:, 1:-1, 1:-1] - I[:-2, 1:-1, 1:-1])]
    w = gaussian_weights(sigma, radius)
    S = {}
    for a in range(3):
        for b in range(a, 3):
            t = g[a] * g[b]
            for axis in (2, 1, 0):
                t = correlate1d(t, w, axis=axis, mode="nearest")
            S[a, b] = t
    det = (S[0, 0] * (S[1, 1] * S[2, 2] - S[1, 2] ** 2) - S[0, 1] * (S[0, 1] * S[2, 2] - S[1, 2] * S[0, 2])
           + S[0, 2] * (S[0, 1] * S[1, 2] - S[1, 1] * S[0, 2]))
    minors = (S[1, 1] * S[2, 2] - S[1, 2] ** 2) + (S[0, 0] * S[2, 2] - S[0, 2] ** 2) + (S[0, 0] * S[1, 1] - S[0, 1] ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(minors > 0, det / minors, 0.0)


def forstner_select(R, mask=None, box=FORSTNER_BOX):
    """(n, 3) voxel positions (x, y, z) of the window maxima of the response R inside mask."""
    from scipy.ndimage import maximum_filter
    Rm = maximum_filter(R, size=box, mode="nearest")     # window offsets -box/2 .. box/2 - 1
    keep = (R == Rm) & (R > 0)
    if mask is not None:
        keep &= np.asarray(mask, dtype=bool)
    z, y, x = np.nonzero(keep)                           # linear index order
    return np.stack([x, y, z], axis=1).astype(np.int64)


def forstner_keypoints(F, mask=None, sigma=FORSTNER_SIGMA, radius=FORSTNER_RADIUS, box=FORSTNER_BOX):
    """Sec. II-C1: keypoints of the fixed image F inside mask."""
    return forstner_select(forstner_response(F, sigma, radius), mask, box)
