"""GB300-native two-level Schwarz neural-operator FGMRES solver for the 2D
frequency-domain Maxwell (Ez) FDFD operator (arXiv 2509.03622).

The compute path lives in the C-ABI library ``libfdfd.so`` (CUDA, sm_103a)
declared in ``include/fdfd.h``; ``paper_2509_03622_gb300.fdfd`` is its thin
ctypes binding.  Importing the binding raises if the library is missing:
there is no CPU fallback.
"""

__all__ = ["fdfd", "workloads"]


def __getattr__(name):
    if name in ("fdfd", "workloads"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
