"""GB300 (sm_103a) DSMC of force-driven rarefied flow between parallel plates: the
micro model of the Micro-Macro-Surrogate method of arXiv 2311.14140.

``Dsmc`` wraps the C ABI of ``include/dsmc.h`` (CUDA kernels in ``csrc/``);
``fields`` turns raw moment sums into cell fields; ``workloads`` names the synthetic
runs.  Build the library with ``__graft_entry__.build()`` or ``_build.build()``.
"""
from .dsmc import Dsmc, DsmcError, Options, default_options, fields, load_library  # noqa: F401

__all__ = ["Dsmc", "DsmcError", "Options", "default_options", "fields", "load_library"]
