"""The autotuner's schedule cache (sfft_autotune_cache), host logic only: a schedule stored
under the problem's key is returned by sfft_autotune without timing anything, and entries
of other problems are kept apart.  On a machine without a GPU the key carries no GPU name,
so the cache is found without any device call."""
import ctypes
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if torch.cuda.is_available():
        pytest.skip("host-only check (with a GPU the key also names the device)")
    from paper_2011_05749_gb300 import _lib
    return _lib.load()


def key(N, f, R, K, n, dtype=0, prec=1, locate=1, noise_auto=0, decoder=0, fma=0):
    return (f"N={N};f={','.join(str(v) for v in f)};R={R};K={K};batch={n};dtype={dtype};"
            f"prec={prec};locate={locate};noise_auto={noise_auto};decoder={decoder};"
            f"fma_only={fma}")


def call(lib, N, f, R, K, n):
    from paper_2011_05749_gb300 import _lib
    base = _lib.Opts()
    lib.sfft_opts_default(ctypes.byref(base))
    f = np.asarray(f, dtype=np.int64)
    delays = np.tile(np.arange(R, dtype=np.int64), (f.size, 1))
    xs = (ctypes.c_void_p * n)(*([8] * n))  # never dereferenced on a cache hit
    best = _lib.Opts()
    rate = ctypes.c_double()
    rc = lib.sfft_autotune(N, K, f.size, f.ctypes.data, R, delays.ctypes.data, ctypes.byref(base),
                           n, ctypes.cast(xs, ctypes.c_void_p), None, ctypes.byref(best),
                           ctypes.byref(rate))
    return rc, best, rate.value


def test_cached_schedule_is_returned(lib, tmp_path):
    path = tmp_path / "tune.json"
    entries = {
        key(2097024, (127, 128, 129), 8, 1000, 256): {"max_tile": 8192, "overlap_gather": 0,
                                                      "classify_lanes": 4, "decode_ctas": 2,
                                                      "rate": 123456.0},
        key(124950, (49, 50, 51), 6, 100, 16): {"max_tile": 0, "overlap_gather": 1,
                                                "classify_lanes": 0, "decode_ctas": 8,
                                                "rate": 5.0},
    }
    path.write_text(json.dumps(entries, indent=1))
    assert lib.sfft_autotune_cache(str(path).encode()) == 0
    rc, best, rate = call(lib, 2097024, (127, 128, 129), 8, 1000, 256)
    assert rc == 0 and rate == 123456.0
    assert (best.max_tile, best.overlap_gather, best.classify_lanes, best.decode_ctas,
            best.max_batch) == (8192, 0, 4, 2, 256)
    rc, best, rate = call(lib, 124950, (49, 50, 51), 6, 100, 16)
    assert rc == 0 and (best.max_tile, best.decode_ctas, rate) == (0, 8, 5.0)
    # a problem that is not in the cache needs the GPU to be timed: an error here, not a hit
    rc, _, _ = call(lib, 124950, (49, 50, 51), 6, 100, 32)
    assert rc != 0
    assert lib.sfft_autotune_cache(None) == 0
