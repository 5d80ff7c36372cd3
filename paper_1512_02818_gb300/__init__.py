"""GB300-native Monte Carlo nodal stage of Probabilistic Domain Decomposition.

The computation lives in the CUDA shared library ``libpdd.so`` (C ABI declared
in ``include/pdd.h``); ``paper_1512_02818_gb300.pdd`` is a thin ctypes binding
with the same function names.  The binding loads the library on first use and
raises if it has not been built -- there is no CPU fallback.
"""
__all__ = ["pdd", "workloads"]
