"""GB300 domain-wall fermion solver: standard and Neff-form 5D operators,
even-odd preconditioned CG with FP64 reliable updates, batched and learned
preconditioned solves.  The compute path is the CUDA library behind the C ABI
in include/dwf.h; ``dwf`` is its ctypes binding and ``inputs`` the seeded
synthetic input generator.  Importing the package loads nothing."""

__all__ = ["dwf", "inputs", "build"]
