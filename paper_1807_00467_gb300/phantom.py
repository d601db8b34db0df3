"""Seeded synthetic lung-CT phantom pairs and test vectors.

This module produces inputs only.  It holds none of the registration
method's arithmetic (no NGF, no interpolation model of the transformation,
no regularisers): both the GPU path and the FP64 oracle receive the arrays
it returns.

Recipe (stands in for the DIR-Lab COPD / 4DCT / EMPIRE10 scans of Sec. III,
which are not available here):

* Volume ``n = (nx, ny, nz)`` voxels of spacing ``h`` mm, cell-centred
  (voxel ``i`` has centre ``(i + 1/2) h``); the field of view is ``n * h``.
* Body: ellipsoid with semi-axes (0.46, 0.40, 0.48) x FOV at +40 HU, air
  -1000 HU outside.
* Lungs: union of two ellipsoids (semi-axes (0.17, 0.26, 0.42) x FOV, centres
  at +-0.20 FOV in x) at -850 HU.
* Vessels: 30 cubic Bezier centre lines with control points inside one lung,
  Gaussian cross-section of radius r ~ U[1, 3] voxels (x spacing), intensity
  -850 + 890 * max_v exp(-d_v^2 / 2 r_v^2) inside the lungs.
* Motion: u*(x) = sum_j A_j exp(-|x - c_j|^2 / (2 * 15^2)), 8 radial basis
  functions with centres uniform in the lung bounding box.  ``motion='small'``:
  A_j uniform in the ball of radius 6 mm.  ``motion='large'``:
  A_j = a (U(-.25,.25), U(-.25,.25), 1), a ~ U(amp_lo, amp_hi) (default 5..20 mm),
  mostly cranio-caudal.  All A_j are scaled by 0.8 until det(I + grad u*) lies
  in [0.25, 4] on a 2 mm lattice.
* Template: T(x + u*(x)) = dens_T(x), where dens_T is the reference density
  with parenchyma raised by 10 % (-850 -> -765 HU).  The inverse map is found
  by Newton's method on a coarse lattice, interpolated to voxels, and dens_T
  is resampled trilinearly at the pre-images.
* Noise: iid Gaussian, sigma 15 HU, independent streams for R and T.
* Keypoints: voxels within one voxel step (max-norm, in voxel units) of the
  voxel nearest to a vessel centre-line sample, inside the lungs, drawn without
  replacement; targets y_KP = x + u*(x) + N(0, sigma_kp^2) per component.

All random numbers come from ``numpy.random.Generator(PCG64)`` streams spawned
from one ``SeedSequence(seed)``.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass, field

import numpy as np

RBF_SIGMA_MM = 15.0


@dataclass
class Phantom:
    R: np.ndarray            # reference (fixed) image, float32 [nz][ny][nx]
    T: np.ndarray            # template (moving) image, float32 [nz][ny][nx]
    n: tuple                 # (nx, ny, nz)
    h: tuple                 # (hx, hy, hz) mm
    amps: np.ndarray         # (8, 3) RBF amplitudes (x, y, z components), mm
    centres: np.ndarray      # (8, 3) RBF centres, mm
    kp_x: np.ndarray | None = None    # (nk, 3) keypoint positions, mm (float32)
    kp_y: np.ndarray | None = None    # (nk, 3) keypoint targets, mm (float32)
    meta: dict = field(default_factory=dict)

    def motion(self, x: np.ndarray) -> np.ndarray:
        """u*(x) for points x (..., 3) in mm."""
        return rbf_motion(x, self.amps, self.centres)


def rbf_motion(x, amps, centres):
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(x.shape, dtype=np.float64)
    s2 = 2.0 * RBF_SIGMA_MM ** 2
    for a, c in zip(amps, centres):
        d2 = np.sum((x - c) ** 2, axis=-1)
        out += np.exp(-d2 / s2)[..., None] * a
    return out


def _rbf_jacobian(x, amps, centres):
    """d u*_i / d x_j at points x (N, 3) -> (N, 3, 3)."""
    x = np.asarray(x, dtype=np.float64)
    diff = x[:, None, :] - np.asarray(centres)[None, :, :]                 # (N, 8, 3)
    e = np.exp(-np.sum(diff * diff, axis=-1) / (2.0 * RBF_SIGMA_MM ** 2))   # (N, 8)
    # d/dx_j exp(-|x-c|^2/(2 s^2)) = -(x_j - c_j)/s^2 * e
    w = diff * (-e / RBF_SIGMA_MM ** 2)[..., None]
    return np.einsum("ki,nkj->nij", np.asarray(amps), w, optimize=True)


def _axis_centres(n, h):
    return (np.arange(n, dtype=np.float64) + 0.5) * h


def _ellipsoid(xc, yc, zc, centre, semi):
    return (((xc - centre[0]) / semi[0]) ** 2 + ((yc - centre[1]) / semi[1]) ** 2
            + ((zc - centre[2]) / semi[2]) ** 2) <= 1.0


def _lung_geometry(fov):
    fov = np.asarray(fov, dtype=np.float64)
    semi = np.array([0.17, 0.26, 0.42]) * fov
    c0 = fov / 2.0
    centres = [c0 + np.array([-0.20 * fov[0], 0.0, 0.0]), c0 + np.array([0.20 * fov[0], 0.0, 0.0])]
    return centres, semi


def _sample_in_ellipsoid(rng, centre, semi, k):
    pts = []
    while len(pts) < k:
        p = rng.uniform(-1.0, 1.0, size=3)
        if np.dot(p, p) <= 1.0:
            pts.append(centre + p * semi)
    return np.array(pts)


def _bezier(ctrl, t):
    t = t[:, None]
    return ((1 - t) ** 3) * ctrl[0] + 3 * ((1 - t) ** 2) * t * ctrl[1] + 3 * (1 - t) * t ** 2 * ctrl[2] + t ** 3 * ctrl[3]


def _vessels(rng, n, h, lung_centres, lung_semi, n_vessels):
    """Rasterise max_v exp(-d_v^2 / 2 r_v^2); returns profile and centre-line samples."""
    nx, ny, nz = n
    hx, hy, hz = h
    prof = np.zeros((nz, ny, nx), dtype=np.float32)
    samples = []
    for _ in range(n_vessels):
        side = rng.integers(0, 2)
        ctrl = _sample_in_ellipsoid(rng, lung_centres[side], 0.85 * lung_semi, 4)
        r_mm = rng.uniform(1.0, 3.0) * hx
        # dense sampling of the centre line: step well below the radius
        approx_len = np.sum(np.linalg.norm(np.diff(ctrl, axis=0), axis=1))
        npts = max(8, int(np.ceil(approx_len / (0.3 * min(r_mm, hx, hy, hz)))))
        pts = _bezier(ctrl, np.linspace(0.0, 1.0, npts))
        samples.append(pts)
        ext = 3.0 * r_mm
        inv2r2 = 1.0 / (2.0 * r_mm * r_mm)
        for p in pts:
            lo = np.floor((p - ext) / np.array(h) - 0.5).astype(int)
            hi = np.ceil((p + ext) / np.array(h) - 0.5).astype(int) + 1
            lo = np.maximum(lo, 0)
            hi = np.minimum(hi, np.array(n))
            if np.any(hi <= lo):
                continue
            xs = (np.arange(lo[0], hi[0]) + 0.5) * hx - p[0]
            ys = (np.arange(lo[1], hi[1]) + 0.5) * hy - p[1]
            zs = (np.arange(lo[2], hi[2]) + 0.5) * hz - p[2]
            d2 = zs[:, None, None] ** 2 + ys[None, :, None] ** 2 + xs[None, None, :] ** 2
            val = np.exp(-d2 * inv2r2).astype(np.float32)
            sl = prof[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
            np.maximum(sl, val, out=sl)
    return prof, samples


def _density(n, h, lung_centres, lung_semi, fov, prof, parenchyma):
    nx, ny, nz = n
    xc = _axis_centres(nx, h[0])[None, None, :]
    yc = _axis_centres(ny, h[1])[None, :, None]
    zc = _axis_centres(nz, h[2])[:, None, None]
    body = _ellipsoid(xc, yc, zc, np.asarray(fov) / 2.0, np.array([0.46, 0.40, 0.48]) * np.asarray(fov))
    lung = _ellipsoid(xc, yc, zc, lung_centres[0], lung_semi) | _ellipsoid(xc, yc, zc, lung_centres[1], lung_semi)
    dens = np.where(body, np.float32(40.0), np.float32(-1000.0)).astype(np.float32)
    lung_val = (parenchyma + (40.0 - parenchyma) * prof).astype(np.float32)
    dens = np.where(lung, lung_val, dens)
    return dens, lung


def _det_range(amps, centres, fov):
    g = [np.arange(1.0, f, 2.0) for f in fov]
    X, Y, Z = np.meshgrid(g[0], g[1], g[2], indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=-1)
    dmin, dmax = np.inf, -np.inf
    for start in range(0, len(pts), 1 << 18):
        J = _rbf_jacobian(pts[start:start + (1 << 18)], amps, centres) + np.eye(3)
        d = (J[:, 0, 0] * (J[:, 1, 1] * J[:, 2, 2] - J[:, 1, 2] * J[:, 2, 1])
             - J[:, 0, 1] * (J[:, 1, 0] * J[:, 2, 2] - J[:, 1, 2] * J[:, 2, 0])
             + J[:, 0, 2] * (J[:, 1, 0] * J[:, 2, 1] - J[:, 1, 1] * J[:, 2, 0]))
        dmin, dmax = min(dmin, float(d.min())), max(dmax, float(d.max()))
    return dmin, dmax


def _inverse_points(z, amps, centres, iters=60, tol=1e-6):
    """Solve x + u*(x) = z for x by Newton's method (points (N, 3)); active-set updates."""
    x = z.copy()
    active = np.arange(len(z))
    for _ in range(iters):
        xa = x[active]
        F = xa + rbf_motion(xa, amps, centres) - z[active]
        keep = np.max(np.abs(F), axis=1) >= tol
        if not np.any(keep):
            break
        active, xa, F = active[keep], xa[keep], F[keep]
        J = _rbf_jacobian(xa, amps, centres) + np.eye(3)
        x[active] = xa - np.linalg.solve(J, F[..., None])[..., 0]
    return x


def _trilinear_upsample(coarse, src_axes, dst_axes):
    """Separable linear interpolation of coarse[(nz,ny,nx, ...)] between lattices."""
    out = coarse
    for ax_idx, axis in ((2, 0), (1, 1), (0, 2)):   # array axis, coordinate axis
        src = src_axes[axis]
        dst = dst_axes[axis]
        pos = np.clip(np.interp(dst, src, np.arange(len(src))), 0, len(src) - 1)
        i0 = np.minimum(np.floor(pos).astype(int), len(src) - 2)
        f = pos - i0
        a = np.take(out, i0, axis=ax_idx)
        b = np.take(out, i0 + 1, axis=ax_idx)
        shape = [1] * out.ndim
        shape[ax_idx] = len(dst)
        f = f.reshape(shape)
        out = a * (1 - f) + b * f
    return out


_RECIPE_VERSION = 1


def make_phantom(n, h, seed, motion="small", amp_range=(5.0, 20.0), n_vessels=30,
                 n_keypoints=0, kp_sigma=1.0, noise_sigma=15.0):
    """Generate a seeded (R, T) phantom pair; see module docstring for the recipe.

    If the environment variable NGF_PHANTOM_CACHE names a directory, phantoms
    are stored there (.npz) and reused by later calls with the same arguments.
    """
    cache = os.environ.get("NGF_PHANTOM_CACHE")
    if cache:
        key = json.dumps([_RECIPE_VERSION, list(n), list(h), int(seed), motion, list(amp_range), n_vessels,
                          n_keypoints, kp_sigma, noise_sigma])
        path = os.path.join(cache, hashlib.sha1(key.encode()).hexdigest()[:16] + ".npz")
        if os.path.exists(path):
            z = np.load(path, allow_pickle=False)
            kx = z["kp_x"] if z["kp_x"].size else None
            ky = z["kp_y"] if z["kp_y"].size else None
            return Phantom(R=z["R"], T=z["T"], n=tuple(int(v) for v in n), h=tuple(float(v) for v in h),
                           amps=z["amps"], centres=z["centres"], kp_x=kx, kp_y=ky, meta=json.loads(str(z["meta"])))
        ph = _make_phantom(n, h, seed, motion, amp_range, n_vessels, n_keypoints, kp_sigma, noise_sigma)
        os.makedirs(cache, exist_ok=True)
        tmp = path + f".{os.getpid()}.npz"
        empty = np.zeros((0, 3), np.float32)
        np.savez(tmp, R=ph.R, T=ph.T, amps=ph.amps, centres=ph.centres,
                 kp_x=ph.kp_x if ph.kp_x is not None else empty, kp_y=ph.kp_y if ph.kp_y is not None else empty,
                 meta=json.dumps(ph.meta))
        os.replace(tmp, path)
        return ph
    return _make_phantom(n, h, seed, motion, amp_range, n_vessels, n_keypoints, kp_sigma, noise_sigma)


def _make_phantom(n, h, seed, motion, amp_range, n_vessels, n_keypoints, kp_sigma, noise_sigma):
    n = tuple(int(v) for v in n)
    h = tuple(float(v) for v in h)
    fov = np.array(n, dtype=np.float64) * np.array(h)
    ss = np.random.SeedSequence(int(seed))
    s_struct, s_noise_r, s_noise_t, s_kp = ss.spawn(4)
    rng = np.random.Generator(np.random.PCG64(s_struct))

    lung_centres, lung_semi = _lung_geometry(fov)
    prof, samples = _vessels(rng, n, h, lung_centres, lung_semi, n_vessels)

    # motion
    lo = np.minimum(lung_centres[0], lung_centres[1]) - lung_semi
    hi = np.maximum(lung_centres[0], lung_centres[1]) + lung_semi
    centres = rng.uniform(lo, hi, size=(8, 3))
    if motion == "small":
        amps = []
        while len(amps) < 8:
            p = rng.uniform(-1.0, 1.0, size=3)
            if np.dot(p, p) <= 1.0:
                amps.append(6.0 * p)
        amps = np.array(amps)
    elif motion == "large":
        a = rng.uniform(amp_range[0], amp_range[1], size=8)
        dirs = np.stack([rng.uniform(-0.25, 0.25, 8), rng.uniform(-0.25, 0.25, 8), np.ones(8)], axis=1)
        amps = a[:, None] * dirs
    else:
        raise ValueError(f"unknown motion {motion!r}")
    rescales = 0
    while True:
        dmin, dmax = _det_range(amps, centres, fov)
        if dmin >= 0.25 and dmax <= 4.0:
            break
        amps = amps * 0.8
        rescales += 1

    dens_R, lung = _density(n, h, lung_centres, lung_semi, fov, prof, -850.0)
    dens_T, _ = _density(n, h, lung_centres, lung_semi, fov, prof, -765.0)

    # pre-images x(z) of template voxel centres, on a coarse lattice (~3 mm)
    coarse_axes = [np.linspace(0.0, f, max(4, int(np.ceil(f / 3.0)) + 1)) for f in fov]
    CZ, CY, CX = np.meshgrid(coarse_axes[2], coarse_axes[1], coarse_axes[0], indexing="ij")
    zc = np.stack([CX, CY, CZ], axis=-1)
    xc = _inverse_points(zc.reshape(-1, 3), amps, centres).reshape(zc.shape)
    disp_c = (xc - zc).astype(np.float64)               # (cz, cy, cx, 3)
    vox_axes = [_axis_centres(n[a], h[a]) for a in range(3)]
    disp = _trilinear_upsample(disp_c, coarse_axes, vox_axes)   # (nz, ny, nx, 3)

    from scipy.ndimage import map_coordinates
    coords = np.empty((3,) + (n[2], n[1], n[0]), dtype=np.float64)
    coords[0] = (vox_axes[2][:, None, None] + disp[..., 2]) / h[2] - 0.5
    coords[1] = (vox_axes[1][None, :, None] + disp[..., 1]) / h[1] - 0.5
    coords[2] = (vox_axes[0][None, None, :] + disp[..., 0]) / h[0] - 0.5
    del disp
    T_clean = map_coordinates(dens_T, coords, order=1, mode="nearest").astype(np.float32)
    del coords

    rng_r = np.random.Generator(np.random.PCG64(s_noise_r))
    rng_t = np.random.Generator(np.random.PCG64(s_noise_t))
    R = dens_R + (noise_sigma * rng_r.standard_normal(dens_R.shape, dtype=np.float32))
    T = T_clean + (noise_sigma * rng_t.standard_normal(T_clean.shape, dtype=np.float32))

    kp_x = kp_y = None
    if n_keypoints > 0:
        rng_k = np.random.Generator(np.random.PCG64(s_kp))
        hv = np.array(h)
        cand = set()
        offs = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)])
        for pts in samples:
            idx = np.round(pts / hv - 0.5).astype(int)
            for base in np.unique(idx, axis=0):
                for ix, iy, iz in base + offs:
                    if 2 <= ix < n[0] - 2 and 2 <= iy < n[1] - 2 and 2 <= iz < n[2] - 2 and lung[iz, iy, ix]:
                        cand.add((ix, iy, iz))
        cand = np.array(sorted(cand), dtype=np.int64)
        k = min(n_keypoints, len(cand))
        pick = cand[rng_k.choice(len(cand), size=k, replace=False)]
        kx = (pick + 0.5) * hv
        ky = kx + rbf_motion(kx, amps, centres) + kp_sigma * rng_k.standard_normal(kx.shape)
        kp_x = kx.astype(np.float32)
        kp_y = ky.astype(np.float32)

    meta = dict(seed=int(seed), motion=motion, rescales=rescales, det_range=[dmin, dmax],
                lung="two ellipsoids", n_vessels=n_vessels, noise_sigma=noise_sigma)
    return Phantom(R=np.ascontiguousarray(R), T=np.ascontiguousarray(T), n=n, h=h,
                   amps=amps, centres=centres, kp_x=kp_x, kp_y=kp_y, meta=meta)


def lung_mask(n, h):
    """uint8 [nz][ny][nx]: 1 inside the two lung ellipsoids of the recipe."""
    fov = np.asarray(n, dtype=np.float64) * np.asarray(h, dtype=np.float64)
    centres, semi = _lung_geometry(fov)
    zc, yc, xc = np.meshgrid(_axis_centres(n[2], h[2]), _axis_centres(n[1], h[1]), _axis_centres(n[0], h[0]),
                             indexing="ij")
    return (_ellipsoid(xc, yc, zc, centres[0], semi) | _ellipsoid(xc, yc, zc, centres[1], semi)).astype(np.uint8)


def node_regions(n, h, m):
    """Boolean [mz][my][mx] masks (body, lungs) of the grid nodes whose support
    (the box of the node's neighbouring cells, [k - 1, k + 1] x node spacing
    per axis, clipped to the field of view) lies inside the body ellipsoid,
    resp. inside one lung ellipsoid of the recipe (both sets are convex, so a
    box is inside when its eight corners are)."""
    fov = np.asarray(n, dtype=np.float64) * np.asarray(h, dtype=np.float64)
    g = fov / (np.asarray(m, dtype=np.float64) - 1.0)
    lo = [np.clip((np.arange(m[a]) - 1.0) * g[a], 0.0, fov[a]) for a in range(3)]
    hi = [np.clip((np.arange(m[a]) + 1.0) * g[a], 0.0, fov[a]) for a in range(3)]
    lung_c, lung_s = _lung_geometry(fov)
    shapes = [(fov / 2.0, np.array([0.46, 0.40, 0.48]) * fov)] + [(c, lung_s) for c in lung_c]
    inside = [np.ones((m[2], m[1], m[0]), dtype=bool) for _ in shapes]
    for cx in (lo[0], hi[0]):
        for cy in (lo[1], hi[1]):
            for cz in (lo[2], hi[2]):
                for k, (c, s) in enumerate(shapes):
                    inside[k] &= _ellipsoid(cx[None, None, :], cy[None, :, None], cz[:, None, None], c, s)
    return inside[0], inside[1] | inside[2]


def _pair_job(job):
    n, h, seed = job
    ph = make_phantom(n, h, seed, motion="large")
    return ph.R, ph.T


def batch_pairs(shapes, seeds, fov=(358.4, 358.4, 320.0), procs=None):
    """[(R, T, h)] for each shape (nx, ny, nz) and seed: independent phantoms
    with large motion (amplitudes U(5, 20) mm) over one field of view, h =
    fov / n.  Made in a pool of spawned processes (safe after the parent has
    initialised CUDA), largest first; a calling script must guard its entry
    point with ``if __name__ == "__main__":`` (spawned children import it)."""
    import multiprocessing as mp
    hs = [tuple(fov[a] / n[a] for a in range(3)) for n in shapes]
    jobs = [(tuple(n), h, int(sd)) for n, h, sd in zip(shapes, hs, seeds)]
    order = sorted(range(len(jobs)), key=lambda i: -int(np.prod(jobs[i][0])))
    procs = procs or max(1, min(len(jobs), os.cpu_count() or 1))
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})   # one thread per child: the pool fills the cores
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_pair_job, [jobs[i] for i in order], chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    out = [None] * len(jobs)
    for k, i in enumerate(order):
        out[i] = (res[k][0], res[k][1], hs[i])
    return out


def motion_on_grid(ph: Phantom, m, scale=1.0) -> np.ndarray:
    """u* sampled at the nodes of an m-node grid spanning the FOV, float32 [3][mz][my][mx]."""
    fov = np.array(ph.n) * np.array(ph.h)
    axes = [np.linspace(0.0, fov[a], m[a]) for a in range(3)]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    u = ph.motion(np.stack([X, Y, Z], axis=-1)) * scale
    return np.ascontiguousarray(np.moveaxis(u, -1, 0).astype(np.float32))


def random_grid_field(m, seed, scale=1.0) -> np.ndarray:
    """N(0, scale^2) mm per component, float32 [3][mz][my][mx]."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    return (scale * rng.standard_normal((3, m[2], m[1], m[0]))).astype(np.float32)


def smooth_grid_field(m, seed, amp=1.0, nmodes=4) -> np.ndarray:
    """A smooth random field (sum of low-frequency cosines), float32 [3][mz][my][mx]."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    axes = [np.linspace(0.0, 1.0, m[a]) for a in range(3)]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    out = np.zeros((3, m[2], m[1], m[0]))
    for c in range(3):
        for _ in range(nmodes):
            k = rng.uniform(0.5, 2.0, size=3)
            ph = rng.uniform(0.0, 2 * np.pi, size=3)
            a = rng.normal() * amp / nmodes
            out[c] += a * np.cos(np.pi * k[0] * X + ph[0]) * np.cos(np.pi * k[1] * Y + ph[1]) * np.cos(np.pi * k[2] * Z + ph[2])
    return out.astype(np.float32)


# Named workloads (voxels, spacing mm, grid nodes, motion).
CONFIGS = {
    "tiny": dict(n=(64, 64, 48), h=(1.0, 1.0, 2.5), m=(17, 17, 13), motion="small"),
    "mid": dict(n=(256, 256, 64), h=(1.4, 1.4, 5.0), m=(65, 65, 33), motion="large"),
    "full": dict(n=(512, 512, 128), h=(0.7, 0.7, 2.5), m=(129, 129, 65), motion="large"),
}
