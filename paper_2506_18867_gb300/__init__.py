"""GB300 (sm_103a) hot path of quadratic B-spline cloth FEM (arXiv 2506.18867).

``bsc`` is the ctypes binding of the C ABI declared in ``include/bsc.h``
(library ``libbsc.so``, built by ``paper_2506_18867_gb300.build``);
``inputs`` draws the seeded synthetic cloth states.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "bsc", "build"]


def __getattr__(name):
    if name in ("bsc", "build"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
