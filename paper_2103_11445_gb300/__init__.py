"""GB300 sparse lower-triangular solver with equation rewriting
(arXiv:2103.11445).

The solver lives in the CUDA library ``libsptrsv.so`` (``csrc/``, C ABI in
``include/sptrsv.h``); :mod:`.binding` is its thin ctypes binding and
:class:`.binding.Plan` a torch-facing wrapper.  Importing this package loads
nothing: the library is loaded (and built from source if absent) on first use.
"""
__all__ = ["binding"]
