"""GB300 (sm_103a) classical and all-floating FETI solver: thin Python binding.

Every numerical step runs in libfeti.so (CUDA kernels behind a C ABI,
declared in include/feti.h); this package only marshals arrays and pointers.
PyTorch tensors may be passed for device input/output buffers.
"""
from .api import FetiError, FetiSolver, checkpoint_read, checkpoint_write, library_path

__all__ = ["FetiError", "FetiSolver", "checkpoint_read", "checkpoint_write", "library_path"]
