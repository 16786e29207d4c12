"""Python front end of libsfft plans, batches and the serving loop (marshalling only)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import check, load, ptr_of, stream_handle


def _torch():
    import torch
    return torch


class Plan:
    """A resident sFFT plan: N, the stages' subsampling factors f (B_d = N / f_d), the
    delays tau_{d,r} (advance sign, [n_stages, R]), the output size K and the options of
    include/sfft.h (sfft_opts)."""

    def __init__(self, N: int, K: int, f, delays, *, dtype: str = "c64",
                 precision: str = "fp32", locate: str = "ml", noise_var: float = 0.0,
                 a_min: float = 1.0, eta: float = 0.0, c0: float = 4.0, c1: float = 2.0,
                 max_rounds: int = 64, max_batch: int = 1, max_tile: int = 0,
                 wait_limit_log2: int = 0, fault_inject: int = 0, decode_ctas: int = 0,
                 decoder: str = "peel", a_m: int = 3, kay_m: int = 2, noise_auto: bool = False,
                 host_gather: bool = False, dft_fma_only: bool = False, dt_method: int = 2,
                 peel_atomic: bool = False, overlap_gather: bool = False,
                 classify_lanes: int = 0, arg_mode: int = 0, ml_tc_tf32: bool = False):
        lib = load()
        f = np.ascontiguousarray(f, dtype=np.int64)
        delays = np.ascontiguousarray(np.asarray(delays, dtype=np.int64).reshape(f.size, -1))
        o = _lib.Opts()
        lib.sfft_opts_default(ctypes.byref(o))
        o.dtype = {"c64": _lib.C64, "c128": _lib.C128}[dtype]
        o.precision = {"fp32": _lib.PREC_FP32, "fp64": _lib.PREC_FP64}[precision]
        o.locate = {"arg": _lib.LOCATE_ARG, "ml": _lib.LOCATE_ML, "kay": _lib.LOCATE_KAY}[locate]
        o.kay_m = kay_m
        o.noise_auto = 1 if noise_auto else 0
        o.host_gather = 1 if host_gather else 0
        o.dft_fma_only = 1 if dft_fma_only else 0
        o.peel_atomic = 1 if peel_atomic else 0
        o.overlap_gather = 1 if overlap_gather else 0
        o.classify_lanes = classify_lanes
        o.arg_mode = arg_mode
        o.ml_tc_tf32 = 1 if ml_tc_tf32 else 0
        o.oneshot_method = dt_method
        o.max_rounds = max_rounds
        o.max_batch = max_batch
        o.max_tile = max_tile
        o.wait_limit_log2 = wait_limit_log2
        o.fault_inject = fault_inject
        o.decode_ctas = decode_ctas
        o.decoder = {"peel": _lib.DECODER_PEEL, "oneshot": _lib.DECODER_ONESHOT,
                     "dsfft": _lib.DECODER_DSFFT}[decoder]
        o.oneshot_am = a_m
        o.noise_var = noise_var
        o.a_min = a_min
        o.eta = eta
        o.c0 = c0
        o.c1 = c1
        h = ctypes.c_void_p()
        check(lib.sfft_plan_create(ctypes.byref(h), N, K, f.size, f.ctypes.data,
                                   delays.shape[1], delays.ctypes.data, ctypes.byref(o)),
              "sfft_plan_create")
        self._h = h
        self.N, self.K = int(N), int(K)
        self.f = tuple(int(v) for v in f)
        self.delays = delays.copy()
        self.R = int(delays.shape[1])
        self.dtype, self.precision, self.locate = dtype, precision, locate
        self.decoder, self.a_m, self.kay_m = decoder, a_m, kay_m
        self.max_batch = max_batch
        self.num_bins = int(lib.sfft_plan_num_bins(h))

    def noise_var(self, slot: int = 0) -> float:
        """sigma^2 estimated for workspace slot `slot` by its last execution (noise_auto)."""
        out = ctypes.c_double()
        check(load().sfft_plan_noise_var(self._h, slot, ctypes.byref(out)), "sfft_plan_noise_var")
        return out.value

    @property
    def handle(self) -> int:
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().sfft_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ outputs
    def _val_dtype(self, torch=None):
        if torch is None:
            return np.complex64 if self.dtype == "c64" else np.complex128
        return torch.complex64 if self.dtype == "c64" else torch.complex128

    def empty_outputs(self, device="cuda", n: int | None = None):
        """(idx int64[K], val complex[K], info int32[4]) buffers on the device (or host
        numpy arrays with device='cpu'), with a leading batch dimension when n is given."""
        shape = (self.K,) if n is None else (n, self.K)
        ishape = (4,) if n is None else (n, 4)
        if device == "cpu":
            return (np.zeros(shape, np.int64), np.zeros(shape, self._val_dtype()),
                    np.zeros(ishape, np.int32))
        torch = _torch()
        return (torch.zeros(shape, dtype=torch.int64, device=device),
                torch.zeros(shape, dtype=self._val_dtype(torch), device=device),
                torch.zeros(ishape, dtype=torch.int32, device=device))

    def execute(self, x, out=None, stream=None):
        """Recover one signal.  x: N complex samples (cuda tensor, or host numpy array /
        cpu tensor, which the library stages through device memory).  Returns
        (idx, val, info) with info = [count, status, rounds, identifications]; entries
        past count are untouched (zero on fresh buffers)."""
        if out is None:
            host = isinstance(x, np.ndarray) or (hasattr(x, "is_cuda") and not x.is_cuda)
            out = self.empty_outputs("cpu" if host else "cuda")
        idx, val, info = out
        check(load().sfft_execute(self._h, ptr_of(x), ptr_of(idx), ptr_of(val), ptr_of(info),
                                  stream_handle(stream)), "sfft_execute")
        return idx, val, info

    def execute_many(self, xs, out=None, stream=None):
        """Recover a batch of signals of this plan (xs: cuda tensor [n, N] or a list)."""
        n = len(xs)
        if out is None:
            out = self.empty_outputs("cuda", n)
        execute_batch([self] * n, list(xs), out, stream)
        return out

    def set_profiling(self, enable: bool = True):
        check(load().sfft_plan_set_profiling(self._h, int(enable)), "sfft_plan_set_profiling")

    def profile(self, reset: bool = True) -> dict:
        """Accumulated CUDA-event time (ms), kernel launches and calls per phase."""
        ms = (ctypes.c_double * 3)()
        la = (ctypes.c_int64 * 3)()
        ca = (ctypes.c_int64 * 3)()
        check(load().sfft_plan_profile(self._h, ms, la, ca, int(reset)), "sfft_plan_profile")
        return {ph: {"ms": ms[i], "launches": la[i], "calls": ca[i]}
                for i, ph in enumerate(("bucketize", "decode", "compact"))}

    def bucketize(self, x, bins=None, stream=None):
        """Bins of Eq. 6 / Eq. 19 in natural order [stage][delay][j] (device only)."""
        torch = _torch()
        if bins is None:
            dt = torch.complex64 if self.precision == "fp32" else torch.complex128
            bins = torch.empty(self.R * self.num_bins, dtype=dt, device=x.device)
        check(load().sfft_bucketize(self._h, ptr_of(x), ptr_of(bins), stream_handle(stream)),
              "sfft_bucketize")
        return bins

    def decode_bins(self, bins, out=None, stream=None):
        """Peeling decoder on caller bins (natural order, arithmetic dtype; device only)."""
        if out is None:
            out = self.empty_outputs("cuda")
        idx, val, info = out
        check(load().sfft_decode_bins(self._h, ptr_of(bins), ptr_of(idx), ptr_of(val),
                                      ptr_of(info), stream_handle(stream)), "sfft_decode_bins")
        return idx, val, info


def execute_batch(plans, xs, out, stream=None):
    """sfft_execute_batch over signals of (possibly) different plans.  out = (idx list,
    val list, infos int32 tensor [n, 4]) or per-plan stacked tensors [n, K]."""
    n = len(plans)
    idx, val, infos = out
    P = ctypes.c_void_p * max(n, 1)
    hp = P(*[p._h.value for p in plans])
    hx = P(*[ptr_of(x) for x in xs])
    hi = P(*[ptr_of(i) for i in idx])
    hv = P(*[ptr_of(v) for v in val])
    check(load().sfft_execute_batch(n, ctypes.cast(hp, ctypes.c_void_p),
                                    ctypes.cast(hx, ctypes.c_void_p),
                                    ctypes.cast(hi, ctypes.c_void_p),
                                    ctypes.cast(hv, ctypes.c_void_p), ptr_of(infos),
                                    stream_handle(stream)), "sfft_execute_batch")
    return out


def autotune(N: int, K: int, f, delays, xs, stream=None, cache: str | None = None, **plan_kw):
    """sfft_autotune: time the schedules on the sample signals xs (device tensors) and return
    (plan keyword arguments of the fastest, its signals/s).  plan_kw as for Plan.  cache: a
    JSON file of schedules found before (sfft_autotune_cache), read and extended."""
    lib = load()
    check(lib.sfft_autotune_cache(cache.encode() if cache else None), "sfft_autotune_cache")
    tmp = Plan(N, K, f, delays, **{**plan_kw, "max_batch": 1})  # validates and fills opts
    o = _lib.Opts()
    lib.sfft_opts_default(ctypes.byref(o))
    o.dtype = {"c64": _lib.C64, "c128": _lib.C128}[tmp.dtype]
    o.precision = {"fp32": _lib.PREC_FP32, "fp64": _lib.PREC_FP64}[tmp.precision]
    o.locate = {"arg": _lib.LOCATE_ARG, "ml": _lib.LOCATE_ML, "kay": _lib.LOCATE_KAY}[tmp.locate]
    o.kay_m = tmp.kay_m
    for k in ("noise_var", "a_min", "eta", "c0", "c1", "max_rounds"):
        if k in plan_kw:
            setattr(o, k, plan_kw[k])
    o.noise_auto = 1 if plan_kw.get("noise_auto") else 0
    o.dft_fma_only = 1 if plan_kw.get("dft_fma_only") else 0
    o.peel_atomic = 1 if plan_kw.get("peel_atomic") else 0
    o.overlap_gather = 1 if plan_kw.get("overlap_gather") else 0
    o.classify_lanes = int(plan_kw.get("classify_lanes", 0))
    tmp.close()
    f = np.ascontiguousarray(f, dtype=np.int64)
    delays = np.ascontiguousarray(np.asarray(delays, dtype=np.int64).reshape(f.size, -1))
    n = len(xs)
    P = ctypes.c_void_p * n
    hx = P(*[ptr_of(x) for x in xs])
    best = _lib.Opts()
    rate = ctypes.c_double()
    check(lib.sfft_autotune(N, K, f.size, f.ctypes.data, delays.shape[1], delays.ctypes.data,
                            ctypes.byref(o), n, ctypes.cast(hx, ctypes.c_void_p),
                            stream_handle(stream), ctypes.byref(best), ctypes.byref(rate)),
          "sfft_autotune")
    kw = dict(plan_kw)
    kw.update(max_batch=best.max_batch, decode_ctas=best.decode_ctas, max_tile=best.max_tile,
              overlap_gather=bool(best.overlap_gather), classify_lanes=best.classify_lanes)
    return kw, rate.value


def bucketize_static(N: int, f, delays, x, bins, precision: str = "fp32",
                     dtype: str = "c64", stream=None) -> int:
    """sfft_bucketize_static: the bins of Eq. 6 / Eq. 19 (natural order, like
    Plan.bucketize) for callers that cannot allocate device memory, so cannot hold a plan.
    x and bins are caller-owned device tensors; the library's fixed 16 MiB device array
    holds everything else.  Returns the C code (SFFT_ETOOBIG when the problem does not fit);
    raises on other errors."""
    f = np.ascontiguousarray(f, dtype=np.int64)
    delays = np.ascontiguousarray(np.asarray(delays, dtype=np.int64).reshape(f.size, -1))
    rc = load().sfft_bucketize_static(
        N, f.size, f.ctypes.data, delays.shape[1], delays.ctypes.data,
        {"fp32": _lib.PREC_FP32, "fp64": _lib.PREC_FP64}[precision],
        {"c64": _lib.C64, "c128": _lib.C128}[dtype], ptr_of(x), ptr_of(bins),
        stream_handle(stream))
    if rc != _lib.SFFT_ETOOBIG:
        check(rc, "sfft_bucketize_static")
    return rc


class Server:
    """Continuous-batching request loop of libsfft (sfft_server_*)."""

    def __init__(self, hbm_budget: int = 8 << 30, max_slots: int = 64):
        h = ctypes.c_void_p()
        check(load().sfft_server_create(ctypes.byref(h), hbm_budget, max_slots),
              "sfft_server_create")
        self._h = h

    def reserve(self, plan: Plan, n: int):
        """sfft_server_reserve: create up to n workspaces for plan's requests now."""
        check(load().sfft_server_reserve(self._h, plan._h, n), "sfft_server_reserve")

    def submit(self, plan: Plan, x, out) -> int:
        idx, val, info = out
        t = ctypes.c_uint64()
        check(load().sfft_submit(self._h, plan._h, ptr_of(x), ptr_of(idx), ptr_of(val),
                                 ptr_of(info), ctypes.byref(t)), "sfft_submit")
        return t.value

    def poll(self, ticket: int):
        """(status, latency_us): status SFFT_PENDING (1) or SFFT_OK (0)."""
        s = ctypes.c_int32()
        lat = ctypes.c_double()
        check(load().sfft_poll(self._h, ticket, ctypes.byref(s), ctypes.byref(lat)), "sfft_poll")
        return s.value, lat.value

    def drain(self):
        check(load().sfft_server_drain(self._h), "sfft_server_drain")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().sfft_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
