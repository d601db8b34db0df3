"""Column-marching GN-product kernel (csrc/gn_product.cu) against the FP64
oracle, and the device-side failure paths (bounded TMA waits, non-finite
objectives) surfacing through rg_sync.

Shapes are chosen to exercise the kernel's variants: cell ratios rho_x in
{2, 4, 8}, rho_y in {2, 4, 8} and rho_z in {1, 2, 4, 8}; volumes whose x and y
extents are not whole tiles; a plane count that is not a whole number of TMA
ring cycles (one column per CTA); and more columns than SMs (persistent CTAs
walking several columns with the plane sequence continued between them).
"""
import numpy as np
import pytest

from helpers import gpu_context, oracle_problem, rel_l2, small_phantom, to_dev

from paper_1807_00467_gb300 import phantom

pytestmark = pytest.mark.gpu

TOL_MV = 1e-5

CASES = [
    ((96, 48, 36), (0.8, 0.8, 2.5), (25, 13, 19)),      # rho (4, 4, 2)
    ((136, 40, 16), (1.0, 1.2, 2.5), (18, 6, 5)),       # rho (8, 8, 4), 136 = 2 x 56 + 24
    ((72, 40, 24), (1.2, 1.2, 2.0), (37, 21, 25)),      # rho (2, 2, 1)
    ((100, 36, 20), (1.0, 1.0, 2.0), (26, 10, 11)),     # rho (4, 4, 2), 3 tile rows (ragged)
    ((68, 24, 32), (1.0, 1.0, 1.5), (18, 7, 5)),        # rho (4, 4, 8)
    ((80, 32, 18), (1.0, 1.0, 2.5), (21, 9, 10)),       # rho (4, 4, 2), 22 planes: one column per CTA
    ((180, 832, 12), (0.9, 0.6, 3.0), (46, 209, 4)),    # rho (4, 4, 4), 156 columns: persistent CTAs
    ((96, 80, 40), (1.0, 1.2, 2.0), (25, 81, 11)),      # rho (4, 1, 4): more box nodes than threads
]


@pytest.mark.parametrize("n,h,m", CASES)
def test_gn_product_against_oracle(n, h, m):
    ph = small_phantom(n, h, seed=11)
    u = phantom.motion_on_grid(ph, m, scale=0.6)
    ctx = gpu_context(ph, m, gamma=0.0)
    ctx.gn_linearize(to_dev(u))
    L = oracle_problem(ph, m, gamma=0.0).linearize(u)
    for seed in (31, 32):
        v = phantom.random_grid_field(m, seed)
        err = rel_l2(ctx.gn_matvec(to_dev(v)).cpu().numpy(), L.matvec(v))
        print(f"{n} rho {[n[a] // (m[a] - 1) for a in range(3)]}: Hv rel-L2 {err:.2e}")
        assert err <= TOL_MV


@pytest.mark.parametrize("n,h,m", [CASES[0], CASES[1], CASES[2], CASES[6]])
def test_pcg_with_column_diagonal_against_oracle(n, h, m):
    """Five PCG steps: the Jacobi diagonal of the NGF term comes from the
    column kernel's diagonal mode, the products from its product mode."""
    ph = small_phantom(n, h, seed=12)
    u = phantom.motion_on_grid(ph, m, scale=0.6)
    ctx = gpu_context(ph, m, gamma=0.001)
    terms, g = ctx.gn_linearize(to_dev(u))
    p, stats = ctx.gn_pcg_solve(g, 5)
    P = oracle_problem(ph, m, gamma=0.001)
    po, so = P.linearize(u).pcg(P.gradient(u)[1], 5)
    assert stats.cpu().numpy()[0] == so[0] == 5
    err = rel_l2(p.cpu().numpy(), po)
    print(f"{n}: 5-step PCG rel-L2 {err:.2e}")
    assert err <= 1e-4


def test_column_kernel_matches_tile_kernel():
    """The column kernel (default) and the tile kernel (general_only through
    tile height 8) agree to FP32 rounding on the same linearisation."""
    n, h, m = CASES[3]
    ph = small_phantom(n, h, seed=13)
    ctx = gpu_context(ph, m, gamma=0.001)
    ctx.gn_linearize(to_dev(phantom.motion_on_grid(ph, m, scale=0.6)))
    v = to_dev(phantom.random_grid_field(m, 33))
    a = ctx.gn_matvec(v).cpu().numpy()
    ctx.set_tile(8)
    b = ctx.gn_matvec(v).cpu().numpy()
    assert rel_l2(a, b) <= 1e-6


def test_bounded_tma_wait_returns_timeout():
    """The GN-product kernels issue no TMA copy (test hook): every bounded wait
    on a TMA barrier runs out, the kernel finishes, and rg_sync reports
    RG_ETIMEOUT; afterwards the context works again."""
    from paper_1807_00467_gb300 import _lib, api
    n, h, m = CASES[0]
    ph = small_phantom(n, h, seed=14)
    u = phantom.motion_on_grid(ph, m, scale=0.6)
    ctx = gpu_context(ph, m, gamma=0.0)
    ctx.gn_linearize(to_dev(u))
    v = to_dev(phantom.random_grid_field(m, 34))
    good = ctx.gn_matvec(v).cpu().numpy()
    assert ctx.sync() == 0
    ctx.debug_hook(_lib.RG_HOOK_POLL_LIMIT, 64)
    ctx.debug_hook(_lib.RG_HOOK_NO_TMA, 1)
    ctx.gn_matvec(v)
    with pytest.raises(api.NgfError) as e:
        ctx.sync()
    assert e.value.code == _lib.RG_ETIMEOUT
    ctx.debug_hook(_lib.RG_HOOK_NO_TMA, 0)
    ctx.debug_hook(_lib.RG_HOOK_POLL_LIMIT, 1 << 20)
    again = ctx.gn_matvec(v).cpu().numpy()
    assert ctx.sync() == 0
    assert np.array_equal(again, good)


@pytest.mark.parametrize("entry", ["objective", "gradient"])
def test_nonfinite_image_is_reported(entry):
    """A NaN in R makes the objective NaN; the asynchronous entry point returns,
    rg_sync reports RG_ENONFINITE, and gn_solve stops with RG_ENONFINITE."""
    import torch

    from paper_1807_00467_gb300 import _lib, api
    n, h, m = CASES[0]
    ph = small_phantom(n, h, seed=15)
    R = ph.R.copy()
    R[n[2] // 2, n[1] // 2, n[0] // 2] = np.nan
    Rd, Td = torch.from_numpy(R).cuda(), torch.from_numpy(ph.T).cuda()
    ctx = api.Context(Rd, Td, ph.h, m, api.make_params(eta=10.0, alpha=1.0))
    u = torch.zeros(ctx.grid_shape, device="cuda")
    terms = ctx.ngf_objective(u) if entry == "objective" else ctx.ngf_gradient(u)[0]
    assert np.isnan(terms.cpu().numpy()[4])
    with pytest.raises(api.NgfError) as e:
        ctx.sync()
    assert e.value.code == _lib.RG_ENONFINITE
    assert ctx.sync() == 0        # the latch is cleared
    with pytest.raises(api.NgfError) as e:
        ctx.gn_solve(u, gn_iters=1, pcg_iters=3)
    assert e.value.code == _lib.RG_ENONFINITE
