"""Seeded synthetic inputs for the aliasing-filter sparse FFT.

This module is shared by the CPU oracle's tests, the CUDA library's tests and the
benchmark.  It holds none of the method's arithmetic: it draws a K-sparse spectrum, turns
it into a time signal (the inverse of Eq. 2, through numpy's FFT), adds white Gaussian
noise at a requested SNR, and draws the random delays the method uses (the random numbers
of R-FFAST are inputs to both implementations, never drawn inside either).

Signal model (Sec. 5.1 of the paper): K distinct frequencies drawn uniformly from [0, N),
each with magnitude 1 (or uniform in [lo, hi]) and a uniformly random phase; the rest of
the spectrum zero, plus, in the general sparse case, complex white Gaussian noise whose
variance sets the SNR:  SNR_dB = 10 log10( sum_n |x_s,n|^2 / sum_n |w_n|^2 ), i.e.
sigma^2 = sum_k |xhat_k|^2 / 10^(SNR/10) per time sample.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Problem:
    N: int
    f: tuple            # subsampling factor L_d of each stage (B_d = N / L_d)
    delays: np.ndarray  # int64 [n_stages, R], advance sign, 0 <= tau < N
    K: int
    support: np.ndarray  # int64 [K], sorted
    values: np.ndarray   # complex128 [K], the paper-normalised xhat at support
    x: np.ndarray        # complex128 [N] time signal (noise included)
    noise_var: float     # sigma^2 per time sample (0 = exactly sparse)
    snr_db: float | None
    seed: int

    @property
    def B(self):
        return tuple(self.N // L for L in self.f)

    @property
    def R(self):
        return int(self.delays.shape[1])


def sparse_spectrum(N: int, K: int, rng: np.random.Generator, mag=(1.0, 1.0)):
    """K distinct uniform frequencies, magnitudes uniform in mag, uniform phase."""
    support = np.sort(rng.choice(N, size=K, replace=False).astype(np.int64))
    lo, hi = mag
    m = np.full(K, lo) if lo == hi else rng.uniform(lo, hi, size=K)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=K)
    return support, m * np.exp(1j * ph)


def time_signal(N: int, support, values) -> np.ndarray:
    """x_n = sum_k xhat_k e^{+2 pi i k n / N}: the inverse of Eq. 2 (numpy ifft carries 1/N)."""
    spec = np.zeros(N, dtype=np.complex128)
    spec[np.asarray(support, dtype=np.int64)] = values
    return np.fft.ifft(spec) * N


def time_signal_torch(N: int, support, values, device="cuda", chunk: int = 1 << 26):
    """The same time signal as time_signal, x_n = sum_k xhat_k e^{+2 pi i k n / N}, built
    directly on a torch device in complex64 for N too large for numpy's FFT: each phase from
    the exact integer residue (k n) mod N, then cos/sin in float64, in chunks of n."""
    import torch
    x = torch.empty(N, dtype=torch.complex64, device=device)
    sup = torch.as_tensor(np.asarray(support, dtype=np.int64), device=device)
    val = torch.as_tensor(np.asarray(values, dtype=np.complex128), device=device)
    two_pi_over_n = 2.0 * math.pi / N
    for n0 in range(0, N, chunk):
        n = torch.arange(n0, min(N, n0 + chunk), dtype=torch.int64, device=device)
        acc = torch.zeros(n.numel(), dtype=torch.complex128, device=device)
        for k, v in zip(sup.tolist(), val.tolist()):
            ph = torch.remainder(n * k, N).to(torch.float64) * two_pi_over_n
            acc += complex(v) * torch.polar(torch.ones_like(ph), ph)
        x[n0:n0 + n.numel()] = acc.to(torch.complex64)
    return x


def noise_variance(values, snr_db) -> float:
    if snr_db is None or math.isinf(snr_db):
        return 0.0
    return float(np.sum(np.abs(values) ** 2) / 10.0 ** (snr_db / 10.0))


def awgn(N: int, var: float, rng: np.random.Generator) -> np.ndarray:
    if var == 0.0:
        return np.zeros(N, dtype=np.complex128)
    s = math.sqrt(var / 2.0)
    return s * rng.standard_normal(N) + 1j * s * rng.standard_normal(N)


def draw_delays(N: int, n_stages: int, R: int, rng: np.random.Generator, fixed=(0, 1)):
    """Per stage: the fixed delays first, then distinct uniform draws from [2, N)."""
    fixed = list(fixed)[:R]
    out = np.zeros((n_stages, R), dtype=np.int64)
    for d in range(n_stages):
        extra = R - len(fixed)
        pick = []
        while len(pick) < extra:
            c = int(rng.integers(2, N))
            if c not in pick and c not in fixed:
                pick.append(c)
        out[d] = fixed + pick
    return out


def kay_delays(N: int, n_stages: int, C: int, m: int, rng: np.random.Generator) -> np.ndarray:
    """Structured R-FFAST delays (Sec. 4.2): per stage, C iterations of m delays
    r_c, r_c + 2^c, ..., r_c + (m - 1) 2^c (mod N) with r_c uniform; slot c m + t.  All
    distinct within a stage."""
    out = np.zeros((n_stages, C * m), dtype=np.int64)
    for d in range(n_stages):
        while True:
            row = []
            for c in range(C):
                r = int(rng.integers(0, N))
                row += [(r + t * (1 << c)) % N for t in range(m)]
            if len(set(row)) == len(row):
                break
        out[d] = row
    return out


def oneshot_delays(N: int, a_m: int, P: int, rng: np.random.Generator) -> np.ndarray:
    """Delays of the one-shot decoder's single stage: the consecutive set -a_m .. 2 a_m - 1
    (mod N), then P distinct uniform draws outside it (Sec. 4.1, Stage 1)."""
    cons = [(k - a_m) % N for k in range(3 * a_m)]
    pick = []
    while len(pick) < P:
        c = int(rng.integers(0, N))
        if c not in pick and c not in cons:
            pick.append(c)
    return np.array([cons + pick], dtype=np.int64)


def make_problem(N, f, K, seed, R=3, delays="ffast", mag=(1.0, 1.0), snr_db=None,
                 support=None, values=None) -> Problem:
    """One seeded problem.  delays="ffast" gives {0, 1, 2} in every stage (Sec. 4.2, exactly
    sparse case); "random" gives 0, 1 and R-2 uniform draws per stage; an array is used as is."""
    rng = np.random.default_rng(seed)
    f = tuple(int(L) for L in f)
    for L in f:
        if N % L:
            raise ValueError(f"L={L} does not divide N={N}")
    if support is None:
        support, values = sparse_spectrum(N, K, rng, mag)
    else:
        support = np.asarray(support, dtype=np.int64)
        values = np.asarray(values, dtype=np.complex128)
        K = support.size
    if isinstance(delays, str):
        if delays == "ffast":
            dl = np.tile(np.arange(R, dtype=np.int64), (len(f), 1))
        elif delays == "random":
            dl = draw_delays(N, len(f), R, rng)
        else:
            raise ValueError(delays)
    else:
        dl = np.asarray(delays, dtype=np.int64).reshape(len(f), -1)
    var = noise_variance(values, snr_db)
    x = time_signal(N, support, values) + awgn(N, var, rng)
    return Problem(N=N, f=f, delays=dl, K=int(K), support=support, values=values, x=x,
                   noise_var=var, snr_db=snr_db, seed=seed)


# Workload shapes of the benchmark configurations (synthetic stand-ins for the paper's
# experiments, Sec. 5.1): N = product of three co-prime factors, B_d = N / f_d.
CONFIGS = {
    # FFAST exactly sparse: N = 20*21*23, delays {0,1,2}, K = 50 unit magnitude
    "ffast_exact_9660": dict(N=9660, f=(20, 21, 23), K=50, R=3, delays="ffast",
                             mag=(1.0, 1.0), snr_db=None),
    # R-FFAST general sparse: N = 127*128*129, 8 delays (0, 1, 6 random), K = 1000,
    # |xhat| ~ U[1,10], SNR 20 dB
    "rffast_2097024": dict(N=2097024, f=(127, 128, 129), K=1000, R=8, delays="random",
                           mag=(1.0, 10.0), snr_db=20.0),
    # mid size used by the batched mix: N = 49*50*51
    "rffast_124950": dict(N=124950, f=(49, 50, 51), K=100, R=6, delays="random",
                          mag=(1.0, 10.0), snr_db=20.0),
    # one-shot decoder (Sec. 3.1, Sec. 4.1 with B = 32 K): N = 2^21, one stage of B = 8192
    # buckets (L = 256), K = 256, a_m = 3, delays -3 .. 5 then 7 random (R = 16)
    "oneshot_2097152": dict(N=2097152, f=(256,), K=256, R=16, delays="oneshot", a_m=3,
                            mag=(1.0, 10.0), snr_db=None),
    # large single signal: N = 511*512*513, 10 delays, K = 10000
    "rffast_134217216": dict(N=134217216, f=(511, 512, 513), K=10000, R=10, delays="random",
                             mag=(1.0, 10.0), snr_db=None),
}


def config_problem(name: str, seed: int, **over) -> Problem:
    c = dict(CONFIGS[name])
    c.update(over)
    delays = c["delays"]
    if delays == "oneshot":
        delays = oneshot_delays(c["N"], c["a_m"], c["R"] - 3 * c["a_m"],
                                np.random.default_rng(seed + 7919))
    return make_problem(c["N"], c["f"], c["K"], seed, R=c["R"], delays=delays,
                        mag=c["mag"], snr_db=c["snr_db"])
