"""GB300-native (sm_103a) subsystem-based ADMM multibody solver.

The solver is the CUDA library ``libsubadmm`` behind the C ABI in ``include/subadmm.h``;
``paper_2302_14344_gb300.subadmm`` is its Python binding and ``paper_2302_14344_gb300.build``
compiles it in-tree.
"""
__all__ = ["build", "subadmm"]
