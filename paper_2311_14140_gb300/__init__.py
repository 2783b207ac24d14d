"""GB300 (sm_103a) DSMC of force-driven rarefied flow between parallel plates: the
micro model of the Micro-Macro-Surrogate method of arXiv 2311.14140.

``Dsmc`` wraps the C ABI of ``include/dsmc.h`` (CUDA kernels in ``csrc/``) for one
run, ``DsmcBatch`` for many independent runs advanced by the same launches,
``DsmcPool`` for runs that come and go (continuous batching, ``DsmcPool.serve``),
``Surrogate`` for the surrogate stage fed by their moment sums, ``mms_hybrid`` for the
MMS hybrid (DSMC in the Knudsen layer, Chapman-Enskog interface, iterated CFD);
``fields`` turns raw moment sums into cell fields; ``workloads`` names the synthetic
runs.  Build the library with ``__graft_entry__.build()`` or ``_build.build()``.
"""
from .dsmc import (Dsmc, DsmcBatch, DsmcError, DsmcPool, GaussianProcess, Options,  # noqa: F401
                   Surrogate, cfd_faces, default_options, fields, load_library, mms_hybrid,
                   solve, surrogate_exponents)

__all__ = ["Dsmc", "DsmcBatch", "DsmcError", "DsmcPool", "GaussianProcess", "Options",
           "Surrogate", "cfd_faces", "default_options", "fields", "load_library", "mms_hybrid",
           "solve", "surrogate_exponents"]
