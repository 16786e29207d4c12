"""CPU checks of the C ABI boundary: libsfft builds, loads without a GPU and exports every
function include/sfft.h declares; the package never reaches the CPU oracle."""
import ast
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sfft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sfft_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("sfft_plan_create", "sfft_execute", "sfft_execute_batch", "sfft_submit",
                 "sfft_poll", "sfft_plan_destroy", "sfft_error_string"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2011_05749_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2011_05749_gb300 import _lib
    assert set(declared_functions()) <= set(_lib.EXPORTS)


def test_error_strings_without_gpu():
    from paper_2011_05749_gb300 import _lib
    lib = _lib.load()
    assert lib.sfft_error_string(0) == b"ok"
    assert b"invalid" in lib.sfft_error_string(-1)


def test_product_code_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2011_05749_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            path = os.path.join(dirpath, fn)
            if fn.endswith(".py"):
                tree = ast.parse(open(path).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        assert not any(a.name.split(".")[0] == "oracle" for a in node.names), path
                    if isinstance(node, ast.ImportFrom):
                        assert (node.module or "").split(".")[0] != "oracle", path
            if fn.endswith((".cu", ".cuh", ".h", ".cpp")):
                assert "sfft_oracle" not in open(path).read(), path


def test_opts_layout_and_defaults_without_gpu():
    """The binding's mirror of sfft_opts matches the C layout: the defaults written by the
    library land in the right fields."""
    import ctypes as ct
    from paper_2011_05749_gb300 import _lib
    o = _lib.Opts()
    for name, _ in _lib.Opts._fields_:
        setattr(o, name, 77)
    _lib.load().sfft_opts_default(ct.byref(o))
    assert (o.dtype, o.precision, o.locate, o.max_rounds, o.max_batch) == (0, 1, 1, 64, 1)
    assert (o.a_min, o.c0, o.c1) == (1.0, 4.0, 2.0)
    assert (o.decoder, o.oneshot_am, o.kay_m, o.noise_auto) == (_lib.DECODER_PEEL, 3, 2, 0)
    assert (o.host_gather, o.oneshot_method, o.dft_fma_only) == (0, 0, 0)
    assert (o.peel_atomic, o.overlap_gather, o.classify_lanes, o.arg_mode, o.ml_tc_tf32) == (0, 0, 0, 0, 0)


def test_schedule_option_ranges_checked_without_gpu():
    """Out-of-range schedule and precision options fail with SFFT_EINVAL before any device
    work: classify_lanes not a power of two up to 32, arg_mode outside 0..3, ml_tc_tf32
    outside {0, 1}."""
    import ctypes as ct
    import numpy as np
    from paper_2011_05749_gb300 import _lib
    lib = _lib.load()
    N, f = 124950, np.array([49, 50, 51], dtype=np.int64)
    delays = np.ascontiguousarray(np.tile(np.arange(3, dtype=np.int64), (3, 1)))

    def create(**kw):
        o = _lib.Opts()
        lib.sfft_opts_default(ct.byref(o))
        for k, v in kw.items():
            setattr(o, k, v)
        h = ct.c_void_p()
        return lib.sfft_plan_create(ct.byref(h), N, 10, 3, f.ctypes.data, delays.shape[1],
                                    delays.ctypes.data, ct.byref(o))
    inval = _lib.SFFT_EINVAL
    assert create(classify_lanes=3) == inval
    assert create(classify_lanes=64) == inval
    assert create(arg_mode=4) == inval
    assert create(ml_tc_tf32=2) == inval
    assert create(ml_tc_tf32=-1) == inval


def test_oneshot_plan_rules_checked_without_gpu():
    """One-shot plans (Sec. 3.1): one stage, K <= B, slots 0 .. 3 a_m - 1 = -a_m .. 2 a_m - 1
    (mod N), at least 2 a_m random delays, Step 2 method 0 (default) .. 3; violations fail
    before any device work."""
    import ctypes as ct
    import numpy as np
    from paper_2011_05749_gb300 import _lib
    lib = _lib.load()
    N, am = 4096, 3
    good = [(k - am) % N for k in range(3 * am)] + [100, 200, 300, 400, 500, 600, 700]

    def create(f, delays, K=10, a_m=am, method=0):
        o = _lib.Opts()
        lib.sfft_opts_default(ct.byref(o))
        o.decoder, o.oneshot_am, o.oneshot_method = _lib.DECODER_ONESHOT, a_m, method
        f = np.ascontiguousarray(f, dtype=np.int64)
        d = np.ascontiguousarray(np.asarray(delays, dtype=np.int64).reshape(f.size, -1))
        h = ct.c_void_p()
        return lib.sfft_plan_create(ct.byref(h), N, K, f.size, f.ctypes.data, d.shape[1],
                                    d.ctypes.data, ct.byref(o))
    inval = _lib.SFFT_EINVAL
    assert create([16, 1], good + good) == inval                      # two stages
    assert create([16], [0] + good[1:]) == inval                      # wrong consecutive set
    assert create([16], good[:13]) == inval                           # P = 4 < 2 a_m
    assert create([16], good, K=N // 16 + 1) == inval                  # K > B
    assert create([16], good, a_m=4) == inval                          # a_m > 3
    assert create([16], good, method=4) == inval                       # Step 2 method 1..3
    assert create([16], good, method=-1) == inval


def test_kay_plan_rules_checked_without_gpu():
    """KAY plans: slot c m + t = r_c + t 2^c (mod N) in every stage and 2^C >= L_d."""
    import ctypes as ct
    import numpy as np
    import synth
    from paper_2011_05749_gb300 import _lib
    lib = _lib.load()
    N, f = 124950, np.array([49, 50, 51], dtype=np.int64)

    def create(delays, m=2):
        o = _lib.Opts()
        lib.sfft_opts_default(ct.byref(o))
        o.locate, o.kay_m = _lib.LOCATE_KAY, m
        d = np.ascontiguousarray(np.asarray(delays, dtype=np.int64).reshape(3, -1))
        h = ct.c_void_p()
        return lib.sfft_plan_create(ct.byref(h), N, 10, 3, f.ctypes.data, d.shape[1],
                                    d.ctypes.data, ct.byref(o))
    inval = _lib.SFFT_EINVAL
    good = synth.kay_delays(N, 3, 6, 2, np.random.default_rng(1))
    bad = good.copy()
    bad[1, 3] = (bad[1, 3] + 1) % N                                  # breaks r_c + 2^c
    assert create(bad) == inval
    assert create(synth.kay_delays(N, 3, 5, 2, np.random.default_rng(1))) == inval  # 2^5 < 51
    assert create(good, m=3) == inval                                # 12 slots, m = 3: wrong structure


def test_noise_auto_rules_checked_without_gpu():
    import ctypes as ct
    import numpy as np
    from paper_2011_05749_gb300 import _lib
    lib = _lib.load()
    N, f = 4096, np.array([16], dtype=np.int64)
    delays = np.ascontiguousarray([[(k - 3) % N for k in range(9)] + [100, 200, 300, 400, 500, 600, 700]],
                                  dtype=np.int64)

    def create(noise_auto, decoder):
        o = _lib.Opts()
        lib.sfft_opts_default(ct.byref(o))
        o.noise_auto, o.decoder = noise_auto, decoder
        h = ct.c_void_p()
        return lib.sfft_plan_create(ct.byref(h), N, 10, 1, f.ctypes.data, delays.shape[1],
                                    delays.ctypes.data, ct.byref(o))
    assert create(2, _lib.DECODER_PEEL) == _lib.SFFT_EINVAL
    assert create(1, _lib.DECODER_ONESHOT) == _lib.SFFT_EINVAL


def test_dsfft_plan_rules_checked_without_gpu():
    """DSFFT plans: N and f[0] powers of two, one stage, delays {0, 1}."""
    import ctypes as ct
    import numpy as np
    from paper_2011_05749_gb300 import _lib
    lib = _lib.load()

    def create(N, L, delays, stages=1):
        o = _lib.Opts()
        lib.sfft_opts_default(ct.byref(o))
        o.decoder = _lib.DECODER_DSFFT
        f = np.ascontiguousarray([L] * stages, dtype=np.int64)
        d = np.ascontiguousarray(np.tile(np.asarray(delays, dtype=np.int64), (stages, 1)))
        h = ct.c_void_p()
        return lib.sfft_plan_create(ct.byref(h), N, 4, stages, f.ctypes.data, d.shape[1],
                                    d.ctypes.data, ct.byref(o))
    inval = _lib.SFFT_EINVAL
    assert create(3000, 8, [0, 1]) == inval          # N not a power of two
    assert create(4096, 12, [0, 1]) == inval         # f[0] not a power of two
    assert create(4096, 8, [0, 2]) == inval          # delays not {0, 1}
    assert create(4096, 8, [0, 1], stages=2) == inval
