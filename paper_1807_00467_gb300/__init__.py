"""GB300 (sm_103a) implementation of the dense continuous registration hot path
of Ruehaak et al., arXiv 1807.00467, Sec. II-D: NGF distance + curvature +
volume change control + keypoint penalty over a trilinear displacement grid,
with matrix-free gradients and Gauss-Newton products, a fixed GN-PCG schedule
and a multilevel driver.

The compute path is libngfreg.so (C ABI in include/ngfreg.h); ``api`` is the
thin torch binding, ``autograd`` puts the objective behind torch.autograd
(backward = the adjoint kernel) and ``phantom`` generates seeded synthetic
inputs.
"""

__version__ = "0.1.0"


def __getattr__(name):
    if name in ("api", "autograd", "phantom", "build"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
