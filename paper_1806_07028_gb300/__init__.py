"""GB300 (sm_103a) implementation of PC-alphaAMG, the path-cover adaptive
unsmoothed-aggregation multigrid method of Hu, Lin and Zikatanov
(arXiv 1806.07028), for weighted graph Laplacians.

The method runs in the CUDA library ``_build/libpcamg.so`` (C ABI in
``include/pcamg.h``); this package is its thin Python binding plus seeded
synthetic inputs. Importing it does not load CUDA; the first call does, and
fails loudly if the library was not built (``build.build()``).
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "Solver", "default_params", "residual", "residual_f32", "uniform",
           "colour", "solve_host", "build", "Mpnn", "training_example", "train", "first_cycles",
           "use_allocator", "allocator_calls"]


def __getattr__(name):
    if name in ("Solver", "default_params", "residual", "residual_f32", "uniform", "colour",
                "solve_host", "Mpnn", "training_example", "train", "first_cycles",
                "use_allocator", "allocator_calls"):
        from . import solver
        return getattr(solver, name)
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
