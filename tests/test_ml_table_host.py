"""Host logic of the first round's ML search on the tensor cores, without a GPU: the table of
A fragments a stage carries (ml_tc_word), read back through the m16n8k8 TF32 A-fragment
layout (lane l, register e: row l / 4 + 8 (e & 1), column l % 4 + 4 (e >> 1) of the 16 x 8
tile), must be the matrix whose product with [Re Z; Im Z] gives
c_q = sum_r Z_r conj(W[r][q]), W[r][q] = e^{2 pi i (q tauL_r mod L) / L} -- computed here
straight from that definition -- for every candidate q < L to within 2^-20 sum_r |Z_r| (rows past L are zero), with both
parts exact TF32 values."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2011_05749_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def probe():
    cxx = shutil.which("g++")
    if not cxx or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("host compiler or CUDA headers missing")
    d = tempfile.mkdtemp()
    exe = os.path.join(d, "ml_table_probe")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-I", CUDA_INC,
                    os.path.join(HERE, "ml_table_probe.cpp"), "-o", exe], check=True)

    def run(L, tauL):
        out = subprocess.run([exe, str(L)] + [str(t) for t in tauL], check=True,
                             capture_output=True, text=True).stdout.split()
        MT, KT = int(out[0]), int(out[1])
        words = np.array([int(w, 16) for w in out[2:]], dtype=np.uint32)
        return MT, KT, words.reshape(MT, KT, 2, 32, 4)
    yield run
    shutil.rmtree(d, ignore_errors=True)


def unpack(MT, KT, words):
    """A (16 MT x 8 KT) from the fragment words, high and low parts."""
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
    return hi, lo


@pytest.mark.parametrize("L,R", [(129, 8), (127, 6), (128, 10), (50, 16), (511, 4), (7, 5)])
def test_ml_table_is_the_candidate_matrix(probe, L, R):
    rng = np.random.default_rng(L * 31 + R)
    tauL = rng.integers(0, L, R)
    MT, KT, words = probe(L, tauL)
    assert MT == (L + 7) // 8 and KT == ((R + 3) // 4 * 4) // 4
    hi, lo = unpack(MT, KT, words)
    # the high part is a TF32 value, the low part the remainder cut to TF32 as well
    assert not np.any(hi.view(np.uint32) & 0x1FFF) and not np.any(lo.view(np.uint32) & 0x1FFF)
    A = hi.astype(np.float64) + lo.astype(np.float64)
    RP = 4 * KT
    Z = rng.standard_normal(R) + 1j * rng.standard_normal(R)
    zv = np.zeros(2 * RP)
    zv[:R], zv[RP:RP + R] = Z.real, Z.imag
    c = A @ zv
    q = np.arange(L)
    W = np.exp(2j * np.pi * ((q[None, :] * tauL[:, None]) % L) / L)  # [r][q]
    ref = (Z[:, None] * np.conj(W)).sum(axis=0)
    got = np.empty(16 * MT // 2, complex)
    for mt in range(MT):
        got[8 * mt:8 * mt + 8] = c[16 * mt:16 * mt + 8] + 1j * c[16 * mt + 8:16 * mt + 16]
    tol = 2.0 ** -20 * np.abs(Z).sum()
    np.testing.assert_allclose(got[:L], ref, rtol=0, atol=tol)
    assert not np.any(got[L:])
