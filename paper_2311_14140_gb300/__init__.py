"""GB300 (sm_103a) DSMC of force-driven rarefied flow between parallel plates: the
micro model of the Micro-Macro-Surrogate method of arXiv 2311.14140.

``Dsmc`` wraps the C ABI of ``include/dsmc.h`` (CUDA kernels in ``csrc/``) for one
run, ``DsmcBatch`` for many independent runs advanced by the same launches;
``fields`` turns raw moment sums into cell fields; ``workloads`` names the synthetic
runs.  Build the library with ``__graft_entry__.build()`` or ``_build.build()``.
"""
from .dsmc import (Dsmc, DsmcBatch, DsmcError, Options, default_options, fields,  # noqa: F401
                   load_library)

__all__ = ["Dsmc", "DsmcBatch", "DsmcError", "Options", "default_options", "fields",
           "load_library"]
