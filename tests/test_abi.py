"""CPU-only checks of the C ABI: the library loads, exports every declared
entry point, and its host-side validation behaves (no kernel is launched)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1807_00467_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "ngfreg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_][a-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ["ngf_objective", "ngf_gradient", "gn_linearize", "gn_matvec", "regularizer_apply",
                 "gn_pcg_solve", "gn_solve", "register_pyramid", "rg_ctx_create", "rg_workspace_size"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1807_00467_gb300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(_lib.EXPORTS)


def test_version_string(lib):
    assert b"sm_103a" in lib.rg_version()


def _geom(n, h, m):
    from paper_1807_00467_gb300._lib import GridGeom, ImageGeom
    ig, gg = ImageGeom(), GridGeom()
    ig.n[:] = n
    ig.h[:] = h
    gg.m[:] = m
    return ig, gg


def test_workspace_size_and_geometry_validation(lib):
    sz = C.c_size_t()
    ig, gg = _geom((512, 512, 128), (0.7, 0.7, 2.5), (129, 129, 65))
    assert lib.rg_workspace_size(C.byref(ig), C.byref(gg), 0, 0, 30, C.byref(sz)) == 0
    N = 512 * 512 * 128
    assert sz.value >= 6 * 4 * N          # stored linearisation a, dT
    assert sz.value < 6 * 4 * N + 2 * 31 * 3 * 4 * 129 * 129 * 65 + 300 * 2 ** 20   # + PCG history
    assert lib.rg_workspace_size(C.byref(ig), C.byref(gg), 0, 0, 64, C.byref(sz)) == -1   # pcg_max > RG_PCG_MAX
    for n, m in [((64, 64, 48), (18, 17, 13)),   # 64 % 17 != 0
                 ((48, 48, 48), (5, 5, 5)),      # rho 12 not a power of two
                 ((3, 64, 48), (2, 17, 13))]:    # too few voxels
        ig, gg = _geom(n, (1.0, 1.0, 1.0), m)
        assert lib.rg_workspace_size(C.byref(ig), C.byref(gg), 0, 0, 30, C.byref(sz)) == -1
    ig, gg = _geom((64, 64, 48), (1.0, -1.0, 1.0), (17, 17, 13))
    assert lib.rg_workspace_size(C.byref(ig), C.byref(gg), 0, 0, 30, C.byref(sz)) == -1
    # the keypoint index: per keypoint its cell, fractions, sorted cell, rank
    # owner and source (36 B), per node the first sorted keypoint of its cell
    # (4 B); at most 2^27 keypoints
    ig, gg = _geom((64, 64, 48), (1.0, 1.0, 1.0), (17, 17, 13))
    s0, s1 = C.c_size_t(), C.c_size_t()
    assert lib.rg_workspace_size(C.byref(ig), C.byref(gg), 0, 0, 30, C.byref(s0)) == 0
    assert lib.rg_workspace_size(C.byref(ig), C.byref(gg), 0, 1000, 30, C.byref(s1)) == 0
    assert s1.value - s0.value >= 36 * 1000 + 4 * 17 * 17 * 13
    assert lib.rg_workspace_size(C.byref(ig), C.byref(gg), 0, 1 << 27, 30, C.byref(sz)) == 0
    assert lib.rg_workspace_size(C.byref(ig), C.byref(gg), 0, (1 << 27) + 1, 30, C.byref(sz)) == -1


def test_context_host_validation(lib):
    from paper_1807_00467_gb300._lib import Params
    ig, gg = _geom((64, 64, 48), (1.0, 1.0, 2.5), (17, 17, 13))
    sz = C.c_size_t()
    assert lib.rg_workspace_size(C.byref(ig), C.byref(gg), 0, 10, 30, C.byref(sz)) == 0
    P = Params(10.0, 1.0, 0.0, 0.0, 0, 10.0)
    ctx = C.c_void_p()
    fake = C.c_void_p(1 << 20)            # never dereferenced on the host
    assert lib.rg_ctx_create(C.byref(ctx), C.byref(ig), C.byref(gg), 0, C.byref(P), 10, 30, fake, sz.value - 1, None) == -1
    assert lib.rg_ctx_create(C.byref(ctx), C.byref(ig), C.byref(gg), 0, C.byref(P), 10, 30, C.c_void_p((1 << 20) + 8),
                             sz.value, None) == -1        # misaligned workspace
    assert lib.rg_ctx_create(C.byref(ctx), C.byref(ig), C.byref(gg), 0, C.byref(P), 10, 30, fake, sz.value, None) == 0
    assert lib.rg_set_keypoints(ctx, 11, fake, fake) == -1   # more than nk_max
    assert b"nk_max" in lib.rg_last_error(ctx)
    bad = Params(-1.0, 1.0, 0.0, 0.0, 0, 10.0)
    assert lib.rg_set_params(ctx, C.byref(bad)) == -1
    assert lib.gn_matvec(ctx, fake, fake) == -1            # no linearisation yet
    assert b"linearisation" in lib.rg_last_error(ctx)
    assert lib.ngf_objective(ctx, None, None) == -1
    assert lib.rg_ctx_destroy(ctx) == 0


def test_pyramid_workspace_validation(lib):
    sz = C.c_size_t()
    ig, gg = _geom((512, 512, 128), (0.7, 0.7, 2.5), (129, 129, 65))
    assert lib.rg_pyramid_workspace_size(C.byref(ig), C.byref(gg), 0, 3, 0, 30, C.byref(sz)) == 0
    one = C.c_size_t()
    lib.rg_workspace_size(C.byref(ig), C.byref(gg), 0, 0, 30, C.byref(one))
    assert one.value < sz.value < 1.5 * one.value
    assert lib.rg_pyramid_workspace_size(C.byref(ig), C.byref(gg), 0, 9, 0, 30, C.byref(sz)) == -1


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1807_00467_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libngfreg.so"))
    with pytest.raises(ImportError):
        _lib.load()
