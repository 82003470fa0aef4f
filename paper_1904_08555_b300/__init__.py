"""Runtime template specialization of numeric CUDA kernels for B300 (sm_103a).

The public surface is the C ABI in include/cj.h (libcj.so); this package is
its Python binding (`cj`) and the build step (`build`).
"""
from . import build  # noqa: F401
from . import cj  # noqa: F401
