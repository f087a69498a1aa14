"""Helpers shared by the tests: run a workload through the oracle or the CUDA binding."""
import numpy as np

TRACE_TOL = 1e-4   # relative L2, GPU FP32 traces vs FP64 oracle
GRAD_TOL = 1e-3    # relative L2 per gradient field


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def oracle_grid(w, **over):
    import oracle
    kw = w.grid_kwargs()
    kw.update(over)
    return oracle.make_grid(**kw)


def gpu_grid(w, **over):
    from paper_1804_01184_gb300 import fwi
    kw = w.grid_kwargs()
    kw.update(over)
    return fwi.make_grid(**kw)
