"""Host logic of the first round's ML search on the tensor cores, without a GPU: each table
of A fragments a stage carries, read back through its MMA's A-fragment layout, must be the
matrix whose product with the bin's [Re Z; Im Z] gives c_q = sum_r Z_r conj(W[r][q]),
W[r][q] = e^{2 pi i (q tauL_r mod L) / L} -- computed here straight from that definition --
for every candidate q < L to within 2^-20 sum_r |Z_r| (rows past L are zero).
  - split TF32 (ml_tc_word, m16n8k8): lane l, register e holds row l / 4 + 8 (e & 1),
    column 8 kt + l % 4 + 4 (e >> 1); columns k < RP take Re Z_k, k >= RP Im Z_{k - RP}
    (RP = R rounded up to 4); both parts exact TF32 values.
  - split FP16 (ml_tc16_word, m16n8k16): lane l, register e holds row l / 4 + 8 (e & 1),
    columns 16 kk + 2 (l % 4) + 8 (e >> 1) + j in half j; column 16 kk + k' takes
    Re Z_{8 kk + k'} (k' < 8) or Im Z_{8 kk + k' - 8}; entries scaled by 2^8, the high part
    the FP16 rounding of the entry."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2011_05749_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"
CASES = [(129, 8), (127, 6), (128, 10), (50, 16), (511, 4), (7, 5), (257, 3)]


@pytest.fixture(scope="module")
def probe():
    cxx = shutil.which("g++")
    if not cxx or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("host compiler or CUDA headers missing")
    d = tempfile.mkdtemp()
    exe = os.path.join(d, "ml_table_probe")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-I", CUDA_INC,
                    os.path.join(HERE, "ml_table_probe.cpp"), "-o", exe], check=True)

    def run(kind, L, tauL):
        out = subprocess.run([exe, kind, str(L)] + [str(t) for t in tauL], check=True,
                             capture_output=True, text=True).stdout.split()
        MT, KT = int(out[0]), int(out[1])
        words = np.array([int(w, 16) for w in out[2:]], dtype=np.uint32)
        return MT, KT, words.reshape(MT, KT, 2, 32, 4)
    yield run
    shutil.rmtree(d, ignore_errors=True)


def reference_scores(L, tauL, Z):
    q = np.arange(L)
    W = np.exp(2j * np.pi * ((q[None, :] * tauL[:, None]) % L) / L)  # [r][q]
    return (Z[:, None] * np.conj(W)).sum(axis=0)


def candidate_values(A, zv, MT):
    c = A @ zv
    got = np.empty(8 * MT, complex)
    for mt in range(MT):
        got[8 * mt:8 * mt + 8] = c[16 * mt:16 * mt + 8] + 1j * c[16 * mt + 8:16 * mt + 16]
    return got


@pytest.mark.parametrize("L,R", CASES)
def test_tf32_table_is_the_candidate_matrix(probe, L, R):
    rng = np.random.default_rng(L * 31 + R)
    tauL = rng.integers(0, L, R)
    MT, KT, words = probe("tf32", L, tauL)
    assert MT == (L + 7) // 8 and KT == (R + 3) // 4
    hi = np.zeros((16 * MT, 8 * KT), np.float32)
    lo = np.zeros_like(hi)
    f = words.view(np.float32)
    for mt in range(MT):
        for kt in range(KT):
            for lane in range(32):
                for e in range(4):
                    row = mt * 16 + lane // 4 + 8 * (e & 1)
                    k = kt * 8 + lane % 4 + 4 * (e >> 1)
                    hi[row, k] = f[mt, kt, 0, lane, e]
                    lo[row, k] = f[mt, kt, 1, lane, e]
    assert not np.any(hi.view(np.uint32) & 0x1FFF) and not np.any(lo.view(np.uint32) & 0x1FFF)
    A = hi.astype(np.float64) + lo.astype(np.float64)
    RP = 4 * KT
    Z = rng.standard_normal(R) + 1j * rng.standard_normal(R)
    zv = np.zeros(2 * RP)
    zv[:R], zv[RP:RP + R] = Z.real, Z.imag
    got = candidate_values(A, zv, MT)
    np.testing.assert_allclose(got[:L], reference_scores(L, tauL, Z), rtol=0,
                               atol=2.0 ** -20 * np.abs(Z).sum())
    assert not np.any(got[L:])


@pytest.mark.parametrize("L,R", CASES)
def test_fp16_table_is_the_candidate_matrix(probe, L, R):
    rng = np.random.default_rng(L * 37 + R)
    tauL = rng.integers(0, L, R)
    MT, KK, words = probe("f16", L, tauL)
    assert MT == (L + 7) // 8 and KK == (R + 7) // 8
    halves = words.view(np.uint16).reshape(MT, KK, 2, 32, 4, 2).view(np.float16)
    hi = np.zeros((16 * MT, 16 * KK), np.float64)
    lo = np.zeros_like(hi)
    for mt in range(MT):
        for kk in range(KK):
            for lane in range(32):
                for e in range(4):
                    for j in range(2):  # j = 0: the low half
                        row = mt * 16 + lane // 4 + 8 * (e & 1)
                        k = kk * 16 + 2 * (lane % 4) + 8 * (e >> 1) + j
                        hi[row, k] = halves[mt, kk, 0, lane, e, j]
                        lo[row, k] = halves[mt, kk, 1, lane, e, j]
    A = (hi + lo) / 2.0 ** 8
    # the high part is the FP16 rounding of the entry: re-rounding hi + lo gives hi back
    np.testing.assert_array_equal((hi + lo).astype(np.float16).astype(np.float64), hi)
    Z = rng.standard_normal(R) + 1j * rng.standard_normal(R)
    zv = np.zeros(16 * KK)
    for r in range(R):
        kk, k = divmod(r, 8)
        zv[16 * kk + k], zv[16 * kk + 8 + k] = Z[r].real, Z[r].imag
    got = candidate_values(A, zv, MT)
    np.testing.assert_allclose(got[:L], reference_scores(L, tauL, Z), rtol=0,
                               atol=2.0 ** -20 * np.abs(Z).sum())
    assert not np.any(got[L:])
