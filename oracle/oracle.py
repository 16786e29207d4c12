"""ctypes front end of ``sfft_oracle.c`` (test infrastructure only).

Every routine here marshals numpy arrays into the C oracle and back; the arithmetic is in
``sfft_oracle.c``, which cites the passages of the paper (Li, Jiang, Chen, arXiv 2011.05749)
it follows.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfft_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/_build/liboracle.so and return its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fcx-limited-range",
           "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("n_recovered", ctypes.c_int32), ("n_out", ctypes.c_int32),
                ("idents", ctypes.c_int64), ("unresolved", ctypes.c_int64),
                ("noise_var", ctypes.c_double)]


class _Opts(ctypes.Structure):
    _fields_ = [("noise_var", ctypes.c_double), ("a_min", ctypes.c_double),
                ("eta", ctypes.c_double), ("c0", ctypes.c_double), ("c1", ctypes.c_double),
                ("locate", ctypes.c_int32), ("max_rounds", ctypes.c_int32),
                ("kay_m", ctypes.c_int32), ("noise_auto", ctypes.c_int32)]


class _RoundLog(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in
                ("idents", "n_zero", "n_single", "n_multi", "n_accepted")]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_oracle())
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int32
            lib.oracle_dense_dft.argtypes = [i64, P, P]
            lib.oracle_bucketize.argtypes = [i64, i32, P, i32, P, P, P, i32]
            lib.oracle_bin.argtypes = [i64, i64, i64, i64, P, P]
            lib.oracle_decode.argtypes = [i64, i32, P, i32, P, P, i32, ctypes.POINTER(_Opts),
                                          P, P, P, P, ctypes.POINTER(_Stats),
                                          ctypes.POINTER(_RoundLog)]
            for fn in (lib.oracle_dense_dft, lib.oracle_bucketize, lib.oracle_bin,
                       lib.oracle_decode):
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def _i64(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=np.int64)


def dense_dft(x) -> np.ndarray:
    """Eq. 1-2 by brute force: xhat_k = (1/N) sum_n x_n e^{-2 pi i k n / N}."""
    x = _c128(x)
    out = np.empty_like(x)
    rc = _load().oracle_dense_dft(x.size, _ptr(x), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_dense_dft failed ({rc})")
    return out


def bucketize(N: int, f, delays, x, n_threads: int | None = None) -> np.ndarray:
    """Eq. 6 / Eq. 19 by naive DFTs.  Returns bins laid out [stage][delay][bin j]."""
    f = _i64(f)
    delays = _i64(delays)
    D = f.size
    R = delays.size // D
    x = _c128(x)
    if x.size != N:
        raise ValueError("x must have N samples")
    total = R * sum(N // int(L) for L in f)
    Y = np.empty(total, dtype=np.complex128)
    nt = n_threads or os.cpu_count() or 1
    rc = _load().oracle_bucketize(N, D, _ptr(f), R, _ptr(delays), _ptr(x), _ptr(Y), nt)
    if rc != 0:
        raise ValueError(f"oracle_bucketize failed ({rc})")
    return Y


def bin_value(N: int, L: int, tau: int, j: int, x) -> complex:
    """One bin Y[j] of the stage with subsampling factor L and delay tau, as a dot product."""
    x = _c128(x)
    out = np.zeros(1, dtype=np.complex128)
    rc = _load().oracle_bin(N, L, tau, j, _ptr(x), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_bin failed ({rc})")
    return complex(out[0])


def gamma_median(R: int) -> float:
    """Median of Gamma(R, 1), the oracle's bisection."""
    lib = _load()
    lib.oracle_gamma_median.restype = ctypes.c_double
    return float(lib.oracle_gamma_median(ctypes.c_int32(R)))


def noise_estimate(N: int, f, R: int, Y) -> float:
    """sigma^2 from the lower median of the bin energies E / B (oracle_noise_estimate)."""
    lib = _load()
    lib.oracle_noise_estimate.restype = ctypes.c_double
    f = _i64(f)
    Y = _c128(Y)
    return float(lib.oracle_noise_estimate(ctypes.c_int64(N), ctypes.c_int32(f.size), _ptr(f),
                                           ctypes.c_int32(R), _ptr(Y)))


@dataclasses.dataclass
class OracleOpts:
    noise_var: float = 0.0
    a_min: float = 1.0
    eta: float = 1e-6
    c0: float = 4.0
    c1: float = 2.0
    locate: int = 0          # 0 ARG (FFAST phase), 1 ML (candidate enumeration), 2 KAY
    max_rounds: int = 64
    kay_m: int = 2           # KAY: delays per iteration (slots c m + t hold r_c + t 2^c)
    noise_auto: int = 0      # 1: sigma^2 from the median bin energy (noise_var unused)


def thresholds(N: int, f, R: int, opts: OracleOpts):
    """(T0_d, T1_d) per stage, the oracle's reading of the unspecified thresholds."""
    out = []
    for L in _i64(f):
        B = N // int(L)
        sig = B * opts.noise_var
        fl = (opts.eta * B * opts.a_min) ** 2
        out.append((R * (opts.c0 * sig + fl), R * (opts.c1 * sig + fl)))
    return out


def decode(N: int, f, delays, Y, K: int, opts: OracleOpts | None = None) -> dict:
    """Peeling decoder (Sec. 3.2) on bins Y (not modified).  Returns a dict with the
    output support/values (sorted by frequency, at most K), every recovered pair in
    acceptance order, the status and per-round counters."""
    opts = opts or OracleOpts()
    f = _i64(f)
    delays = _i64(delays)
    D = f.size
    R = delays.size // D
    Y = _c128(Y).copy()
    nb = sum(N // int(L) for L in f)
    out_idx = np.zeros(max(K, 1), dtype=np.int64)
    out_val = np.zeros(max(K, 1), dtype=np.complex128)
    rec_f = np.zeros(nb, dtype=np.int64)
    rec_v = np.zeros(nb, dtype=np.complex128)
    mr = opts.max_rounds
    logs = {k: np.zeros(mr, dtype=np.int64)
            for k in ("idents", "n_zero", "n_single", "n_multi", "n_accepted")}
    rl = _RoundLog(*[_ptr(logs[k]) for k in
                     ("idents", "n_zero", "n_single", "n_multi", "n_accepted")])
    co = _Opts(opts.noise_var, opts.a_min, opts.eta, opts.c0, opts.c1, opts.locate, mr, opts.kay_m,
               opts.noise_auto)
    st = _Stats()
    rc = _load().oracle_decode(N, D, _ptr(f), R, _ptr(delays), _ptr(Y), K, ctypes.byref(co),
                               _ptr(out_idx), _ptr(out_val), _ptr(rec_f), _ptr(rec_v),
                               ctypes.byref(st), ctypes.byref(rl))
    if rc != 0:
        raise ValueError(f"oracle_decode failed ({rc})")
    n = st.rounds
    return {
        "idx": out_idx[: st.n_out].copy(),
        "val": out_val[: st.n_out].copy(),
        "rec_f": rec_f[: st.n_recovered].copy(),
        "rec_v": rec_v[: st.n_recovered].copy(),
        "status": st.status,
        "rounds": st.rounds,
        "idents": st.idents,
        "unresolved": st.unresolved,
        "noise_var": st.noise_var,
        "round_log": {k: v[:n].copy() for k, v in logs.items()},
    }
