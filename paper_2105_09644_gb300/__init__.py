"""GB300 (sm_103a) implementation of the TreeRay/OnTheSpot hot path.

The compute path is the CUDA library ``libtreeray.so`` (sources in
``csrc/``, C ABI in ``include/treeray.h``); ``binding`` is its ctypes
front end.  ``build()`` compiles the library in-tree.
"""
import importlib


def build(force: bool = False, verbose: bool = False) -> str:
    from .buildlib import build as _build
    return _build(force=force, verbose=verbose)


def __getattr__(name):
    if name == "binding":
        return importlib.import_module(".binding", __name__)
    raise AttributeError(name)
