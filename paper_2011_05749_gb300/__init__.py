"""GB300 (sm_103a) aliasing-filter sparse FFT with peeling decoding (FFAST / R-FFAST).

Li, Jiang, Chen, "On Performance of Sparse Fast Fourier Transform Algorithms Using the
Aliasing Filter" (arXiv 2011.05749), Sec. 2-4.  The computation lives in libsfft (CUDA,
C ABI in include/sfft.h); this package is its thin Python binding.

    plan = Plan(N, K, f=(127, 128, 129), delays=delays, noise_var=s2, max_batch=64)
    idx, val, info = plan.execute(x)          # x: complex64 cuda tensor of N samples
"""
from .plan import Plan, Server, autotune, bucketize_static, execute_batch  # noqa: F401
from ._lib import SfftError, load, library_path  # noqa: F401
from . import _lib  # noqa: F401
