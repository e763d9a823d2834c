"""GB300 CentRA sample-and-cover (Pellegrina, KDD'23, Algorithm 1) on one GPU.

The method runs in libcen.so (include/cen.h), hand-written CUDA for sm_103a;
``paper_2306_03651_gb300.cen`` is its ctypes binding and the names it exports
(``Graph``, ``Job``, ``run``, ``bounds``, the raw ``cen_*`` entry points) are
reachable from this package.  ``paper_2306_03651_gb300.inputs`` holds the
seeded synthetic graph generators and does not load the CUDA library.
"""
import importlib

_SUBMODULES = ("cen", "inputs", "serve", "tune", "_build")


def __getattr__(name):
    if name in _SUBMODULES:
        return importlib.import_module(f"{__name__}.{name}")
    if name.startswith("__"):
        raise AttributeError(name)
    cen = importlib.import_module(f"{__name__}.cen")
    try:
        return getattr(cen, name)
    except AttributeError:
        raise AttributeError(f"module {__name__!r} has no attribute {name!r}") from None
