"""GB300-native reduced-speed-of-light radiative transfer on Voronoi meshes.

The hot path (upwind transport + implicit comoving source step, Sec. 2.2 and
2.3 of Chang, Davis & Jiang) runs in the CUDA library librt_gb300.so behind
the C ABI of include/rt.h; this package holds its Python binding
(capi, solver), the build step and the seeded input generators (inputs).
Importing the package does not load the CUDA library.
"""
__all__ = ["RTSolver"]


def __getattr__(name):
    if name == "RTSolver":
        from .solver import RTSolver
        return RTSolver
    raise AttributeError(name)
