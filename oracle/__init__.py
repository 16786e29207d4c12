"""FP64 CPU oracle for the aliasing-filter sparse FFT (FFAST / R-FFAST peeling).

Test infrastructure only: the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg use it to check and time the CUDA library.  The library never imports it,
and it imports nothing from the library.
"""
from .oracle import (  # noqa: F401
    build_oracle,
    dense_dft,
    bucketize,
    bin_value,
    decode,
    OracleOpts,
    thresholds,
    gamma_median,
    noise_estimate,
)
