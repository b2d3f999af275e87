"""GB300-native (sm_103a) hot path of Bayesian multidimensional scaling fitted
by Hamiltonian Monte Carlo (Holbrook et al., arXiv:1905.04582).

- ``capi``: ctypes binding of the C ABI in ``include/mds.h``.
- ``mds``: ``MDS`` context object and the ``MDSLogLik`` autograd function.
- ``workloads``: seeded synthetic inputs shaped like the paper's workloads.
- ``build``: in-tree nvcc build of ``_lib/libmds.so``.

Importing the package does not load the CUDA library; the first ``MDS(...)``
does, and raises if it was not built.
"""
__all__ = ["capi", "mds", "workloads", "build"]


def __getattr__(name):
    import importlib
    if name in __all__:
        return importlib.import_module(f".{name}", __name__)
    if name in ("MDS", "MDSLogLik", "mds_loglik"):
        return getattr(importlib.import_module(".mds", __name__), name)
    raise AttributeError(name)
