"""DSFFT: the iterative framework's binary tree search (Sec. 3.3, Sec. 4.3), FP64.

TEST INFRASTRUCTURE ONLY: the CUDA library never imports this module.

N = 2^n.  Layer d of the tree holds the 2^d nodes y_{2^d,0}[i] = sum_{f = i mod 2^d} xhat_f
(Eq. 23 up to the factor B = 2^d): the aliasing-filter bins of subsampling factor
L = N / 2^d.  Subproblem 1 computes a layer selectively or all at once by an FFT; here every
layer is computed whole, by numpy's FFT of the stride-L subsample (a library primitive for
one step).  The search starts at layer p (O(log K), Sec. 3.3) and goes down one layer at a
time.  Subproblem 2 (stopping): the search ends at the first layer where every efficient
node holds one frequency -- m_d = K in the exactly sparse case -- or at the last layer.
Subproblem 3 (recovery in each single-frequency bucket): the phase encoding of Sec. 3.2
with delays {0, 1}, i.e. the peeling decoder of sfft_oracle.c on one stage with ARG locate
(one stage cannot peel a multi-frequency bucket, so a layer with one is "not finished").
m_d, the number of efficient nodes, is the number of bins that are not zero-tons.

Pinned by tests/test_oracle_pins.py: the paper's N = 64 example (layer counts 1, 2, 4, 5,
stop at d = 3, the five frequencies) and exact recovery of the truth.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import oracle as core


def layer_bins(x: np.ndarray, N: int, d: int) -> np.ndarray:
    """Bins [delay tau in {0, 1}][i < 2^d] of layer d: the B-point DFT of x[tau::L]."""
    B = 1 << d
    L = N // B
    x = np.asarray(x, dtype=np.complex128)
    return np.concatenate([np.fft.fft(x[tau::L][:B]) for tau in (0, 1)])


@dataclasses.dataclass
class DsfftResult:
    idx: np.ndarray
    val: np.ndarray
    status: int              # 0 when the stop layer's nodes were all single-frequency
    stop_layer: int
    layer_counts: list       # m_d of every layer searched, from the start layer on


def decode(N: int, K: int, x, start_layer: int, opts: core.OracleOpts | None = None,
           last_layer: int | None = None) -> DsfftResult:
    """The search from start_layer down to last_layer (default log2 N)."""
    n = N.bit_length() - 1
    if 1 << n != N:
        raise ValueError("N must be a power of two")
    if last_layer is not None:
        n = min(n, last_layer)
    opts = opts or core.OracleOpts()
    opts = dataclasses.replace(opts, locate=0)
    counts = []
    res = None
    d = start_layer
    for d in range(start_layer, n + 1):
        B = 1 << d
        Y = layer_bins(x, N, d)
        res = core.decode(N, [N // B], [[0, 1]], Y, K, opts)
        counts.append(int(B - res["round_log"]["n_zero"][0]))
        if res["status"] == 0:
            break
    return DsfftResult(idx=res["idx"], val=res["val"], status=int(res["status"]), stop_layer=d,
                       layer_counts=counts)
