"""GB300-native (sm_103a) Scheme III hot path of arXiv:1804.01184.

Time-domain staggered-grid finite-difference modelling of the 2-D variable-density acoustic
wave equation: forward shots (``fwi_model``), Born modelling (``fwi_born``), and adjoint
back-propagation with the zero-lag cross-correlation fused into the gradient for all five
parameterizations of Table 1 (``fwi_adjoint``, ``fwi_gradient``).  The compute path is the
CUDA library ``libfwi.so`` (C ABI declared in ``include/fwi.h``); ``paper_1804_01184_gb300.fwi``
is its thin Python binding.  ``inputs`` holds the seeded synthetic workloads.  ``fborn`` binds
the frequency-domain Born path of the paper's Schemes I/II (analytic Green functions, Born
data, misfit gradient, Hessian column); ``engine``, ``serve``, ``autograd``, ``bowls``,
``invert`` and ``dist`` build on the library calls.

The binding is imported lazily so that ``inputs`` can be used without a GPU.
"""
import importlib

__all__ = ["fwi", "inputs"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
