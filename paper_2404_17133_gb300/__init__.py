"""GB300 rid-preconditioned Davidson solver for TDDFT response problems (arXiv 2404.17133).

The solver is the CUDA library built from ``csrc/`` (C ABI in include/tddft.h);
``api`` is its Python binding.  Import ``paper_2404_17133_gb300.api`` after
``paper_2404_17133_gb300.build.build()`` has produced the library.
"""
__all__ = ["build", "api"]
