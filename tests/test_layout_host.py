"""Host logic of the bucketization layout (pfa_layout.h), without a GPU: a small probe
program built with the host compiler lays out single stages and reports their axes.

Checked: which odd axes take the tensor-core path (FP32 stages done in one pass, odd
17 <= P <= 127, none when allow_tc is off, none in FP64 or two-pass stages), the twiddle
table offsets (consecutive, 16-byte aligned, fragment tables of 2 KB per row tile and
k-tile), the shared-memory budget (tensor-core tables stay out of it) and the prime-factor
strides."""
import json
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2011_05749_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"
SMEM = 232448  # opt-in shared memory per block of the target GPU


@pytest.fixture(scope="module")
def probe():
    cxx = shutil.which("g++")
    if not cxx or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("host compiler or CUDA headers missing")
    d = tempfile.mkdtemp()
    exe = os.path.join(d, "layout_probe")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", CSRC, "-I", CUDA_INC,
                    os.path.join(HERE, "layout_probe.cpp"), "-o", exe], check=True)

    def run(B, esz=8, allow_tc=1, max_tile=0):
        out = subprocess.run([exe, str(B), str(esz), str(SMEM), str(allow_tc), str(max_tile)],
                             check=True, capture_output=True, text=True).stdout
        return json.loads(out)
    yield run
    shutil.rmtree(d, ignore_errors=True)


def mtiles(P):
    return ((P + 1) // 2 + 15) // 16


def ktiles(P):
    return ((P + 1) // 2 + 31) // 32 * 4


def odd_tc(P):
    return P % 2 == 1 and 17 <= P <= 127


@pytest.mark.parametrize("B", [16512, 16383, 16256, 2550, 2499, 2450, 6806, 6723, 6642])
def test_one_pass_fp32_stages_take_tensor_core_odd_axes(probe, B):
    lay = probe(B)
    assert lay["ok"] and not lay["two_pass"]
    prod = 1
    for ax in lay["axes"]:
        prod *= ax["P"]
        assert ax["tc"] == (1 if (not ax["pow2"] and odd_tc(ax["P"])) else 0), ax
    assert prod == B


@pytest.mark.parametrize("B", [16512, 16383, 16256])
def test_no_tensor_core_axes_when_disallowed_or_fp64(probe, B):
    for lay in (probe(B, allow_tc=0), probe(B, esz=16)):
        assert lay["ok"]
        assert all(ax["tc"] == 0 for ax in lay["axes"])


@pytest.mark.parametrize("B", [262656, 262143, 261632])
def test_two_pass_stages_keep_fma_axes(probe, B):
    lay = probe(B)
    assert lay["ok"] and lay["two_pass"]
    assert all(ax["tc"] == 0 for ax in lay["axes"])
    assert 0 < lay["split"] < len(lay["axes"])


@pytest.mark.parametrize("B,allow", [(16383, 1), (16383, 0), (16512, 1), (2499, 1)])
def test_twiddle_offsets_and_sizes(probe, B, allow):
    """Axes' twiddles are laid out back to back from 0, each block even-sized (16-byte
    aligned in FP32); a tensor-core axis holds mtiles * ktiles / 2 fragment tiles of 2 KB
    (256 entries of 8 bytes: m16n8k16 tiles of 16 inputs, two 8-row groups each)."""
    lay = probe(B, allow_tc=allow)
    off = 0
    for ax in lay["axes"]:
        assert ax["tw_off"] == off and off % 2 == 0
        P = ax["P"]
        if ax["tc"]:
            n = mtiles(P) * (ktiles(P) // 2) * 256
        elif ax["pow2"]:
            n = P // 2
        else:
            pairs = (P - 1) // 2
            gp = 1 if pairs <= 1 else 2 if pairs <= 2 else 4 if pairs <= 4 else 8
            n = pairs * ((pairs + gp - 1) // gp * gp)
        off += n + (n & 1)
    assert lay["tw_total"] == off


def test_large_odd_tables_stay_out_of_shared_memory(probe):
    """The one-pass launch's shared memory holds the tile plus the radix-2 and small odd
    axes' twiddles only: B = 16383 (127, 43, 3) needs the tile and the 3-point table, with
    tensor-core axes or without (the 127- and 43-point tables are read from global memory
    either way)."""
    with_tc, without = probe(16383), probe(16383, allow_tc=0)
    tile = (16383 + 1) * 8
    assert with_tc["smem1"] == tile + 2 * 8  # the 3-point table: one pair row of 2
    assert without["smem1"] == with_tc["smem1"]
    # B = 16512 (43, 3, 128): the 3-point table and the 64 radix-2 twiddles
    assert probe(16512)["smem1"] == (16512 + 64 + 2) * 8


@pytest.mark.parametrize("B", [16512, 16383, 2550])
def test_strides_are_prime_factor_products(probe, B):
    lay = probe(B)
    S = 1
    for ax in lay["axes"]:
        assert ax["S"] == S
        S *= ax["P"]
    assert S == B
