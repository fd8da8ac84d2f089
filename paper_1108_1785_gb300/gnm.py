"""Python binding of libgnm.so (the C ABI declared in include/gnm.h).

Argument marshalling only: every step of the flow analysis runs in the library's CUDA
kernels. Device buffers are torch CUDA tensors (their data_ptr() is passed through),
streams are torch streams. The library must have been built (``build.build()``); the
binding raises if it is missing instead of computing anything itself.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GNM_CHECKED=1 in the environment selects the build with device-side bounds checks
LIB_PATH = os.path.join(_HERE, "libgnm_checked.so" if os.environ.get("GNM_CHECKED") == "1" else "libgnm.so")

NO_SITE = 0xFFFFFFFF
NSTAT = 6
LOOKUP_AUTO, LOOKUP_BSEARCH, LOOKUP_RMI, LOOKUP_RADIX, LOOKUP_HASH24 = 0, 1, 2, 3, 4
PLACE_AUTO, PLACE_SMEM, PLACE_L2, PLACE_STAGED = 0, 1, 2, 3
AGG_AUTO, AGG_DIRECT, AGG_WARP = 0, 1, 2
ADMIN_OR, ADMIN_AND = 0, 1
TABLE_AUTO, TABLE_DIRECT, TABLE_HASH, TABLE_GLOBAL, TABLE_PARTITION = 0, 1, 2, 3, 4
SPLIT_AUTO, SPLIT_FUSED, SPLIT_TWO_KERNELS = 0, 1, 2
ROOT_LINEAR, ROOT_MLP = 0, 1
FIT_MINIMAX, FIT_MSE = 0, 1
DEBUG_RMI_SPLIT_BASE = 1
HOST_AUTO, HOST_STAGE, HOST_IN_PLACE, HOST_PIPELINE = 0, 1, 2, 3
RATE_BUCKETS = 10001
NO_MEDIAN = 0xFFFFFFFF
KERNEL_TIMES = 1  # GNM_PLAN_KERNEL_TIMES
KERNEL_NAMES = {0: "k_keys", 1: "k_aggregate", 2: "k_finalize_windows", 3: "k_part_count", 4: "k_part_scan",
                5: "k_part_scatter"}
FIELDS = ("srcaddr", "dstaddr", "dPkts", "dOctets", "first", "last")

STATUS = {0: "GNM_OK", 1: "GNM_E_INVAL", 2: "GNM_E_NOMEM", 3: "GNM_E_CUDA", 4: "GNM_E_STATE",
          5: "GNM_E_CAPACITY", 6: "GNM_E_TIMEOUT", 7: "GNM_E_INTERNAL"}


class GnmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("min_avg_pkt_bytes", C.c_uint32), ("min_pkts", C.c_uint32), ("min_dur_ms", C.c_uint32),
                ("min_flows_to_flag", C.c_uint32), ("admin_rule", C.c_int32), ("lookup_mode", C.c_int32),
                ("placement", C.c_int32), ("aggregation", C.c_int32), ("device", C.c_int32),
                ("window_slots", C.c_uint32), ("threshold_bps", C.c_double), ("block_threads", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("unroll", C.c_int32), ("table_mode", C.c_int32),
                ("hash_slots", C.c_uint32), ("radix_bits", C.c_uint32), ("split", C.c_int32),
                ("key_directory", C.c_int32), ("host_records", C.c_int32), ("rate_stats", C.c_int32),
                ("host_capacity", C.c_uint32)]


class RecordsC(C.Structure):
    _fields_ = [("n", C.c_uint64)] + [(f, C.c_void_p) for f in FIELDS] + \
        [("srcport", C.c_void_p), ("dstport", C.c_void_p), ("prot", C.c_void_p), ("on_device", C.c_int32)]


class SiteStat(C.Structure):
    _fields_ = [("site", C.c_uint32), ("dir", C.c_uint32), ("flows", C.c_uint64), ("octets", C.c_uint64),
                ("pkts", C.c_uint64), ("e_flows", C.c_uint64), ("e_octets", C.c_uint64),
                ("e_dur_ms", C.c_uint64), ("rate_bps", C.c_double), ("flag", C.c_uint32),
                ("reserved", C.c_uint32)]


class RegistryInfo(C.Structure):
    _fields_ = [("n_ranges", C.c_uint64), ("n_registered", C.c_uint64), ("n_sites", C.c_uint32),
                ("n_prefixes", C.c_uint32), ("placement", C.c_int32), ("lookup_mode", C.c_int32),
                ("privatized", C.c_int32), ("rmi_ready", C.c_int32)]


class RmiConfig(C.Structure):
    _fields_ = [("root_kind", C.c_int32), ("n_leaves", C.c_uint32), ("hidden", C.c_uint32),
                ("leaf_iters", C.c_uint32), ("mlp_steps", C.c_uint32), ("mlp_batch", C.c_uint32),
                ("mlp_lr", C.c_float), ("seed", C.c_uint32), ("exhaustive_eps", C.c_int32),
                ("leaf_fit", C.c_int32), ("eps_target", C.c_uint32), ("max_split_log2", C.c_uint32)]


class RmiReport(C.Structure):
    _fields_ = [("n_train", C.c_uint64), ("root_loss", C.c_double), ("leaf_loss", C.c_double),
                ("eps_max", C.c_uint32), ("err_max", C.c_uint32), ("eps_mean", C.c_double),
                ("empty_leaves", C.c_uint32), ("n_models", C.c_uint32), ("split_leaves", C.c_uint32),
                ("train_ms", C.c_double), ("sweep_ms", C.c_double)]


class StreamConfig(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("n_cuda_streams", C.c_uint32), ("max_queued", C.c_uint32),
                ("max_batch_records", C.c_uint64)]


class WindowDone(C.Structure):
    _fields_ = [("window_id", C.c_uint64), ("records", C.c_uint64), ("latency_ms", C.c_double),
                ("status", C.c_int32), ("reserved", C.c_int32), ("queued_ms", C.c_double)]


class StreamStats(C.Structure):
    _fields_ = [("batches", C.c_uint64), ("batches_queued", C.c_uint64), ("records", C.c_uint64),
                ("windows_closed", C.c_uint64), ("windows_done", C.c_uint64), ("inflight_bytes", C.c_uint64),
                ("peak_inflight_bytes", C.c_uint64), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("max_ms", C.c_double), ("mean_ms", C.c_double)]


class HostStat(C.Structure):
    _fields_ = [("addr", C.c_uint32), ("site", C.c_uint32), ("dir", C.c_uint32), ("reserved", C.c_uint32),
                ("flows", C.c_uint64), ("octets", C.c_uint64), ("pkts", C.c_uint64), ("e_flows", C.c_uint64),
                ("e_octets", C.c_uint64), ("e_dur_ms", C.c_uint64), ("rate_bps", C.c_double)]


class TuneReport(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("ctas_per_sm", C.c_int32), ("unroll", C.c_int32),
                ("aggregation", C.c_int32), ("placement", C.c_int32), ("best_ms", C.c_double),
                ("default_ms", C.c_double), ("n_tried", C.c_uint32), ("radix_bits", C.c_uint32),
                ("split", C.c_int32), ("key_directory", C.c_int32), ("keys_unroll", C.c_int32),
                ("best_ms_by_agg", C.c_double * 3)]


_lib = None


def checked_build() -> bool:
    """True when the loaded library is the build with device-side bounds checks."""
    return bool(lib().gnm_checked_build())


def lib():
    """The loaded C library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1108_1785_gb300.build.build() first "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        P, S, U64, U32 = C.c_void_p, C.c_size_t, C.c_uint64, C.c_uint32
        st = C.c_int
        sig = {
            "gnm_config_default": (None, [C.POINTER(Config)]),
            "gnm_create": (st, [C.POINTER(Config), C.POINTER(P)]),
            "gnm_destroy": (None, [P]),
            "gnm_last_error": (C.c_char_p, [P]),
            "gnm_registry_load": (st, [P, P, P, P, S, U32, P, P, S]),
            "gnm_registry_info_get": (st, [P, C.POINTER(RegistryInfo)]),
            "gnm_registry_ranges": (st, [P, P, P, S, C.POINTER(S)]),
            "gnm_registry_flatten": (st, [P, P, P, S, U32, P, P, S, C.POINTER(S)]),
            "gnm_window_process": (st, [P, C.POINTER(RecordsC), U64, P]),
            "gnm_windows_process": (st, [P, C.POINTER(RecordsC), P, P, S, P]),
            "gnm_window_open": (st, [P, U64, P]),
            "gnm_window_add": (st, [P, C.POINTER(RecordsC), U64, P]),
            "gnm_window_close": (st, [P, U64, P]),
            "gnm_window_export": (st, [P, U64, P, S, C.POINTER(S)]),
            "gnm_window_import": (st, [P, U64, P, S, P]),
            "gnm_site_stats": (st, [P, U64, C.POINTER(SiteStat), S, C.POINTER(S), P]),
            "gnm_flag_suboptimal": (st, [P, U64, C.c_double, P, P, S, C.POINTER(S)]),
            "gnm_window_dense": (st, [P, U64, P, P, P, P]),
            "gnm_window_device": (st, [P, U64, C.POINTER(P), C.POINTER(P), C.POINTER(P)]),
            "gnm_windows_results": (st, [P, P, S, P, P, P, P]),
            "gnm_windows_results_async": (st, [P, P, S, P, P, P, P, P]),
            "gnm_window_release": (st, [P, U64]),
            "gnm_lookup": (st, [P, P, U64, P, P, P]),
            "gnm_rates": (st, [P, P, U64, P, P]),
            "gnm_rmi_config_default": (None, [C.POINTER(RmiConfig)]),
            "gnm_rmi_train": (st, [P, P, U64, C.POINTER(RmiConfig), C.POINTER(RmiReport), P]),
            "gnm_rmi_violations": (st, [P, C.POINTER(U64), C.c_int]),
            "gnm_rmi_linear_grad": (st, [P, P, P, U64, C.c_float, C.c_float, P, P]),
            "gnm_rmi_mlp_grad": (st, [P, P, P, U64, U32, P, P, P]),
            "gnm_rmi_export": (st, [P, P, P, P, P, P, P, P, P, P, P]),
            "gnm_rmi_import": (st, [P, C.c_int32, U32, U32, P, P, P, P, P, P]),
            "gnm_plan_create": (st, [P, C.POINTER(RecordsC), P, P, S, C.POINTER(P)]),
            "gnm_plan_launch": (st, [P, P]),
            "gnm_plan_create_ex": (st, [P, C.POINTER(RecordsC), P, P, S, U32, C.POINTER(P)]),
            "gnm_plan_kernel_times": (st, [P, P, P, S, C.POINTER(S)]),
            "gnm_plan_destroy": (None, [P]),
            "gnm_autotune": (st, [P, C.POINTER(RecordsC), P, P, S, C.POINTER(TuneReport)]),
            "gnm_last_launch_count": (U32, [P]),
            "gnm_window_rate_stats": (st, [P, U64, P, P, P, P]),
            "gnm_window_rate_cells": (st, [P, U64, P, P, P, C.c_size_t, C.POINTER(C.c_size_t)]),
            "gnm_checked_build": (C.c_int, []),
            "gnm_device_checks": (st, [P, C.POINTER(U64)]),
            "gnm_debug_corrupt": (st, [P, C.c_int32, U32, U32]),
            "gnm_warnings_update": (st, [P, U64, U32, U32, P, S, C.POINTER(S)]),
            "gnm_warnings_reset": (st, [P]),
            "gnm_warnings_export": (st, [P, P]),
            "gnm_warnings_import": (st, [P, P]),
            "gnm_window_hosts": (st, [P, U64, P, S, C.POINTER(S)]),
            "gnm_stream_config_default": (None, [C.POINTER(StreamConfig)]),
            "gnm_stream_open": (st, [P, C.POINTER(StreamConfig), C.POINTER(P)]),
            "gnm_stream_submit": (st, [P, C.POINTER(RecordsC), U64, C.c_int]),
            "gnm_stream_poll": (st, [P, C.POINTER(WindowDone), S, C.POINTER(S), C.c_int]),
            "gnm_stream_submit_many": (st, [P, C.POINTER(RecordsC), P, P, P, P, S, C.POINTER(S)]),
            "gnm_stream_stats_get": (st, [P, C.POINTER(StreamStats)]),
            "gnm_stream_close": (None, [P]),
            "gnm_window_process_noalloc": (st, [C.POINTER(Config), P, P, U32, U32, P, P, S, C.POINTER(RecordsC),
                                                P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(ctx_ptr, status: int):
    if status != 0:
        msg = lib().gnm_last_error(ctx_ptr)
        raise GnmError(status, msg.decode() if msg else "")


def _ptr(a) -> int:
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Records:
    """A struct-of-arrays record batch: six uint32 arrays, all torch CUDA tensors
    (device) or all numpy arrays (host). Keeps the arrays alive while in use."""

    def __init__(self, fields: Dict[str, object]):
        self.fields = {k: fields[k] for k in FIELDS}
        first = self.fields["srcaddr"]
        self.on_device = hasattr(first, "data_ptr") and getattr(first, "is_cuda", False)
        n = {int(v.numel() if hasattr(v, "numel") else v.size) for v in self.fields.values()}
        if len(n) != 1:
            raise ValueError("record arrays differ in length")
        self.n = n.pop()
        for k, v in self.fields.items():
            dt = str(v.dtype)
            if "int32" not in dt:  # torch.int32 or numpy uint32 / int32
                raise TypeError(f"{k} must hold 32-bit integers, got {dt}")
            if hasattr(v, "is_contiguous") and not v.is_contiguous():
                raise ValueError(f"{k} must be contiguous")
        self.c = RecordsC()
        self.c.n = self.n
        for k in FIELDS:
            setattr(self.c, k, _ptr(self.fields[k]))
        self.c.on_device = 1 if self.on_device else 0

    @staticmethod
    def to_device(rec: Dict[str, np.ndarray], device: str = "cuda") -> "Records":
        import torch
        return Records({k: torch.from_numpy(np.ascontiguousarray(rec[k]).view(np.int32)).to(device)
                        for k in FIELDS})

    @staticmethod
    def host(rec: Dict[str, np.ndarray]) -> "Records":
        return Records({k: np.ascontiguousarray(rec[k], dtype=np.uint32) for k in FIELDS})


def registry_flatten(prefix, plen, site, n_sites: int) -> Tuple[np.ndarray, np.ndarray]:
    """Host-only registry flattening (no GPU): sorted range starts and their sites."""
    p = np.ascontiguousarray(prefix, np.uint32)
    l = np.ascontiguousarray(plen, np.uint8)
    s = np.ascontiguousarray(site, np.uint32)
    n = C.c_size_t()
    st = lib().gnm_registry_flatten(_ptr(p), _ptr(l), _ptr(s), p.size, n_sites, None, None, 0, C.byref(n))
    if st not in (0, 5):
        _check(None, st)
    a = np.empty(n.value, np.uint32)
    b = np.empty(n.value, np.uint32)
    _check(None, lib().gnm_registry_flatten(_ptr(p), _ptr(l), _ptr(s), p.size, n_sites, _ptr(a), _ptr(b),
                                            n.value, C.byref(n)))
    return a, b


def rates(e_octets, e_dur_ms, rate, stream=None):
    """The rate step alone (gnm_rates): rate[i] = e_octets[i] * 8000 / e_dur_ms[i] as the window
    calls compute it, for device uint64 tensors of sums and a float64 device tensor."""
    n = int(e_octets.numel())
    if int(e_dur_ms.numel()) != n or int(rate.numel()) < n:
        raise ValueError("e_octets, e_dur_ms and rate need n entries")
    _check(None, lib().gnm_rates(_ptr(e_octets), _ptr(e_dur_ms), n, _ptr(rate), _stream_ptr(stream)))


def window_process_noalloc(starts, site, n_sites: int, local_prefix, local_len, rec: "Records", stats, rate, flag,
                           stream=None, **cfg):
    """One window without any device allocation by the library (gnm_window_process_noalloc):
    the caller provides the flattened registry (device starts/site), device records and
    device result arrays stats[(2*n_sites+4)*6] (u64), rate[2*n_sites] (f64), flag[2*n_sites]."""
    c = Config()
    lib().gnm_config_default(C.byref(c))
    for k, v in cfg.items():
        if not hasattr(c, k):
            raise TypeError(f"unknown config key {k}")
        setattr(c, k, v)
    lp = np.ascontiguousarray(local_prefix, np.uint32)
    ll = np.ascontiguousarray(local_len, np.uint8)
    _check(None, lib().gnm_window_process_noalloc(C.byref(c), _ptr(starts), _ptr(site), int(starts.numel()), n_sites,
                                                  _ptr(lp), _ptr(ll), lp.size, C.byref(rec.c), _ptr(stats), _ptr(rate),
                                                  _ptr(flag), _stream_ptr(stream)))


class Context:
    """A gnm context (one GPU)."""

    def __init__(self, **cfg):
        L = lib()
        c = Config()
        L.gnm_config_default(C.byref(c))
        for k, v in cfg.items():
            if not hasattr(c, k):
                raise TypeError(f"unknown config key {k}")
            setattr(c, k, v)
        self.config = c
        h = C.c_void_p()
        _check(None, L.gnm_create(C.byref(c), C.byref(h)))
        self.h = h
        self.n_sites = 0

    def close(self):
        if getattr(self, "h", None):
            lib().gnm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _c(self, status):
        _check(self.h, status)

    # ---------------------------------------------------------------- registry
    def load_registry(self, prefix, plen, site, n_sites: int, local_prefix, local_len):
        p = np.ascontiguousarray(prefix, np.uint32)
        l = np.ascontiguousarray(plen, np.uint8)
        s = np.ascontiguousarray(site, np.uint32)
        lp = np.ascontiguousarray(local_prefix, np.uint32)
        ll = np.ascontiguousarray(local_len, np.uint8)
        self._c(lib().gnm_registry_load(self.h, _ptr(p), _ptr(l), _ptr(s), p.size, n_sites, _ptr(lp),
                                        _ptr(ll), lp.size))
        self.n_sites = n_sites

    def load(self, reg):
        """Registry object with prefix/plen/site/n_sites/local_prefix/local_len."""
        self.load_registry(reg.prefix, reg.plen, reg.site, reg.n_sites, reg.local_prefix, reg.local_len)

    def registry_info(self) -> RegistryInfo:
        info = RegistryInfo()
        self._c(lib().gnm_registry_info_get(self.h, C.byref(info)))
        return info

    def ranges(self) -> Tuple[np.ndarray, np.ndarray]:
        n = C.c_size_t()
        lib().gnm_registry_ranges(self.h, None, None, 0, C.byref(n))
        st = np.empty(n.value, np.uint32)
        si = np.empty(n.value, np.uint32)
        self._c(lib().gnm_registry_ranges(self.h, _ptr(st), _ptr(si), n.value, C.byref(n)))
        return st, si

    # ---------------------------------------------------------------- windows
    def process(self, rec: Records, window_id: int, stream=None):
        self._c(lib().gnm_window_process(self.h, C.byref(rec.c), window_id, _stream_ptr(stream)))

    def process_windows(self, rec: Records, offsets: Sequence[int], window_ids: Sequence[int], stream=None):
        off = np.ascontiguousarray(offsets, np.uint64)
        ids = np.ascontiguousarray(window_ids, np.uint64)
        self._c(lib().gnm_windows_process(self.h, C.byref(rec.c), _ptr(off), _ptr(ids), ids.size,
                                          _stream_ptr(stream)))

    def open(self, window_id: int, stream=None):
        self._c(lib().gnm_window_open(self.h, window_id, _stream_ptr(stream)))

    def add(self, rec: Records, window_id: int, stream=None):
        self._c(lib().gnm_window_add(self.h, C.byref(rec.c), window_id, _stream_ptr(stream)))

    def close_window(self, window_id: int, stream=None):
        self._c(lib().gnm_window_close(self.h, window_id, _stream_ptr(stream)))

    def window_export(self, window_id: int) -> np.ndarray:
        """The sums an open window holds so far: (2*n_sites + 4, 6) uint64 rows (flows,
        octets, pkts, e_flows, e_octets, e_dur_ms), site keys then the unmatched classes."""
        n = C.c_size_t()
        st = lib().gnm_window_export(self.h, window_id, None, 0, C.byref(n))
        if st != 5:  # GNM_E_CAPACITY: the size is in n
            self._c(st)
        rows = np.empty((n.value, 6), np.uint64)
        self._c(lib().gnm_window_export(self.h, window_id, _ptr(rows), n.value, C.byref(n)))
        return rows

    def window_import(self, window_id: int, rows, stream=None):
        """Opens `window_id` with `rows` (as window_export gives them) as its sums so far."""
        r = np.ascontiguousarray(rows, np.uint64)
        self._c(lib().gnm_window_import(self.h, window_id, _ptr(r), r.shape[0], _stream_ptr(stream)))

    def release(self, window_id: int):
        self._c(lib().gnm_window_release(self.h, window_id))

    def dense(self, window_id: int):
        """(stats[2S, 6] u64, unmatched[4, 3] u64, rate[2S] f64, flag[2S] u8) on the host."""
        nk = 2 * self.n_sites
        st = np.empty((nk, NSTAT), np.uint64)
        un = np.empty((4, 3), np.uint64)
        r = np.empty(nk, np.float64)
        f = np.empty(nk, np.uint8)
        self._c(lib().gnm_window_dense(self.h, window_id, _ptr(st), _ptr(un), _ptr(r), _ptr(f)))
        return st, un, r, f

    def windows_results(self, window_ids, stats=None, unmatched=None, rate=None, flag=None):
        """Dense results of many windows into caller-provided host arrays (one sync)."""
        ids = np.ascontiguousarray(window_ids, np.uint64)
        self._c(lib().gnm_windows_results(self.h, _ptr(ids), ids.size, _ptr(stats), _ptr(unmatched), _ptr(rate),
                                          _ptr(flag)))

    def windows_results_async(self, window_ids, stats=None, unmatched6=None, rate=None, flag=None, stream=None):
        """gnm_windows_results_async: the copies enqueued on `stream` (default: torch's
        current stream); the host arrays (page-locked) are valid after it synchronises.
        unmatched6: [n][4][NSTAT] u64, the unmatched rows as stored."""
        ids = np.ascontiguousarray(window_ids, np.uint64)
        self._c(lib().gnm_windows_results_async(self.h, _ptr(ids), ids.size, _ptr(stats), _ptr(unmatched6),
                                                _ptr(rate), _ptr(flag), _stream_ptr(stream)))

    def device_checks(self) -> int:
        """The checked build's error word since the last call (0: no failed bounds check);
        raises GnmError (GNM_E_INTERNAL) when a check failed."""
        w = C.c_uint64()
        self._c(lib().gnm_device_checks(self.h, C.byref(w)))
        return w.value

    def debug_corrupt(self, what: int, index: int, value: int):
        """Checked build only: overwrite one value of the device state (see gnm.h)."""
        self._c(lib().gnm_debug_corrupt(self.h, what, index, value))

    def rate_cells(self, window_id: int):
        """Non-empty cells of a finalised window's rate histograms: (key, bucket, count)
        arrays in (key, bucket) order (rate_stats = 1 or 2)."""
        n = C.c_size_t()
        st = lib().gnm_window_rate_cells(self.h, window_id, None, None, None, 0, C.byref(n))
        if st not in (0, 5):
            self._c(st)
        k = np.empty(n.value, np.uint32)
        b = np.empty(n.value, np.uint32)
        c = np.empty(n.value, np.uint32)
        self._c(lib().gnm_window_rate_cells(self.h, window_id, _ptr(k), _ptr(b), _ptr(c), n.value, C.byref(n)))
        return k, b, c

    def rate_stats(self, window_id: int, hist: bool = False):
        """(rmin[2S], rmax[2S], median_bucket[2S], hist[2S, 10001] or None) of a finalised
        window of a context made with rate_stats=1 (dense histograms) or 2 (sparse: no
        dense histogram, see rate_cells)."""
        nk = 2 * self.n_sites
        rmin = np.empty(nk, np.float64)
        rmax = np.empty(nk, np.float64)
        med = np.empty(nk, np.uint32)
        h = np.empty((nk, RATE_BUCKETS), np.uint32) if hist else None
        self._c(lib().gnm_window_rate_stats(self.h, window_id, _ptr(rmin), _ptr(rmax), _ptr(med), _ptr(h)))
        return rmin, rmax, med, h

    def hosts(self, window_id: int):
        """Per-host rows of a window: (addr u32, site u32, dir u8, sums[n, 6] u64, rate f64),
        sorted by (site, dir, addr)."""
        n = C.c_size_t()
        st = lib().gnm_window_hosts(self.h, window_id, None, 0, C.byref(n))
        if st not in (0, 5):
            self._c(st)
        buf = (HostStat * max(n.value, 1))()
        self._c(lib().gnm_window_hosts(self.h, window_id, buf, n.value, C.byref(n)))
        a = np.frombuffer(buf, dtype=np.dtype([(f, np.uint32) for f in ("addr", "site", "dir", "reserved")] +
                                             [(f, np.uint64) for f in ("flows", "octets", "pkts", "e_flows",
                                                                       "e_octets", "e_dur_ms")] +
                                             [("rate_bps", np.float64)]), count=n.value)
        sums = np.stack([a[f] for f in ("flows", "octets", "pkts", "e_flows", "e_octets", "e_dur_ms")], axis=1)
        return a["addr"].copy(), a["site"].copy(), a["dir"].astype(np.uint8), sums, a["rate_bps"].copy()

    def warnings_update(self, window_id: int, below_bucket: int = 100, consecutive: int = 2) -> np.ndarray:
        """Keys (site*2+dir) warned about after this window (the next one in time order)."""
        out = np.empty(2 * self.n_sites, np.uint32)
        n = C.c_size_t()
        self._c(lib().gnm_warnings_update(self.h, window_id, below_bucket, consecutive, _ptr(out), out.size,
                                          C.byref(n)))
        return out[:n.value].copy()

    def warnings_reset(self):
        self._c(lib().gnm_warnings_reset(self.h))

    def warnings_export(self) -> np.ndarray:
        runs = np.empty(2 * self.n_sites, np.uint32)
        self._c(lib().gnm_warnings_export(self.h, _ptr(runs)))
        return runs

    def warnings_import(self, runs):
        r = np.ascontiguousarray(runs, np.uint32)
        if r.size != 2 * self.n_sites:
            raise ValueError("runs must have 2 * n_sites entries")
        self._c(lib().gnm_warnings_import(self.h, _ptr(r)))

    def device_results(self, window_id: int):
        """Raw device addresses (stats, rate, flag) of a window's dense results."""
        a, b, c = C.c_void_p(), C.c_void_p(), C.c_void_p()
        self._c(lib().gnm_window_device(self.h, window_id, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def site_stats(self, window_id: int):
        n = C.c_size_t()
        un = np.empty(12, np.uint64)
        s = lib().gnm_site_stats(self.h, window_id, None, 0, C.byref(n), _ptr(un))
        if s not in (0, 5):
            self._c(s)
        arr = (SiteStat * max(n.value, 1))()
        self._c(lib().gnm_site_stats(self.h, window_id, arr, n.value, C.byref(n), _ptr(un)))
        return [arr[i] for i in range(n.value)], un.reshape(4, 3)

    def flag_suboptimal(self, window_id: int, threshold_bps: float):
        n = C.c_size_t()
        cap = 2 * self.n_sites
        sites = np.empty(cap, np.uint32)
        dirs = np.empty(cap, np.uint8)
        self._c(lib().gnm_flag_suboptimal(self.h, window_id, threshold_bps, _ptr(sites), _ptr(dirs), cap,
                                          C.byref(n)))
        return sites[:n.value].copy(), dirs[:n.value].copy()

    def lookup(self, addr, site_out=None, pos_out=None, stream=None):
        """Longest-prefix match of a device uint32 tensor of addresses."""
        self._c(lib().gnm_lookup(self.h, _ptr(addr), int(addr.numel()), _ptr(site_out), _ptr(pos_out),
                                 _stream_ptr(stream)))

    def last_launch_count(self) -> int:
        return int(lib().gnm_last_launch_count(self.h))

    # ------------------------------------------------------------ learned index
    def rmi_train(self, keys, stream=None, **cfg) -> RmiReport:
        c = RmiConfig()
        lib().gnm_rmi_config_default(C.byref(c))
        for k, v in cfg.items():
            setattr(c, k, v)
        rep = RmiReport()
        self._c(lib().gnm_rmi_train(self.h, _ptr(keys), int(keys.numel()), C.byref(c), C.byref(rep),
                                    _stream_ptr(stream)))
        return rep

    def rmi_violations(self, reset: bool = False) -> int:
        v = C.c_uint64()
        self._c(lib().gnm_rmi_violations(self.h, C.byref(v), int(reset)))
        return v.value

    def rmi_linear_grad(self, z, y, w: float, c: float, stream=None) -> np.ndarray:
        g = np.zeros(3, np.float64)
        self._c(lib().gnm_rmi_linear_grad(self.h, _ptr(z), _ptr(y), int(z.numel()), w, c, _ptr(g),
                                          _stream_ptr(stream)))
        return g

    def rmi_mlp_grad(self, xn, y, hidden: int, params: np.ndarray, stream=None) -> np.ndarray:
        p = np.ascontiguousarray(params, np.float32)
        g = np.zeros(3 * hidden + 2, np.float64)
        self._c(lib().gnm_rmi_mlp_grad(self.h, _ptr(xn), _ptr(y), int(xn.numel()), hidden, _ptr(p), _ptr(g),
                                       _stream_ptr(stream)))
        return g

    def rmi_export(self):
        """The learned index: root parameters, per-leaf split words and per-model lines and
        error bounds (models: the leaves, then the sub-leaves of split leaves)."""
        kind = C.c_int32()
        L = C.c_uint32()
        M = C.c_uint32()
        self._c(lib().gnm_rmi_export(self.h, C.byref(kind), C.byref(L), C.byref(M), None, None, None, None, None,
                                     None, None))
        n, m = L.value, M.value
        root = np.zeros(2 + 3 * 32 + 1, np.float32)
        split = np.zeros(n, np.uint32)
        a = np.zeros(m, np.float32)
        b = np.zeros(m, np.float32)
        x0 = np.zeros(m, np.uint32)
        elo = np.zeros(m, np.uint32)
        ehi = np.zeros(m, np.uint32)
        self._c(lib().gnm_rmi_export(self.h, C.byref(kind), C.byref(L), C.byref(M), _ptr(root), _ptr(split), _ptr(a),
                                     _ptr(b), _ptr(x0), _ptr(elo), _ptr(ehi)))
        return dict(root_kind=kind.value, n_leaves=n, n_models=m, root=root, split=split, a=a, b=b, x0=x0,
                    eps_lo=elo, eps_hi=ehi)

    def rmi_import(self, root_kind: int, root, a, b, x0, split=None, n_leaves=None, stream=None):
        r = np.ascontiguousarray(root, np.float32)
        a = np.ascontiguousarray(a, np.float32)
        b = np.ascontiguousarray(b, np.float32)
        x0 = np.ascontiguousarray(x0, np.uint32)
        sp = None if split is None else np.ascontiguousarray(split, np.uint32)
        L = int(n_leaves) if n_leaves is not None else (sp.size if sp is not None else a.size)
        self._c(lib().gnm_rmi_import(self.h, root_kind, L, a.size, _ptr(r), _ptr(sp),
                                     _ptr(a), _ptr(b), _ptr(x0), _stream_ptr(stream)))

    # ---------------------------------------------------------- plans / tuning
    def plan(self, rec: Records, offsets, window_ids, kernel_times: bool = False) -> "Plan":
        return Plan(self, rec, offsets, window_ids, kernel_times)

    def autotune(self, rec: Records, offsets, window_ids) -> TuneReport:
        off = np.ascontiguousarray(offsets, np.uint64)
        ids = np.ascontiguousarray(window_ids, np.uint64)
        rep = TuneReport()
        self._c(lib().gnm_autotune(self.h, C.byref(rec.c), _ptr(off), _ptr(ids), ids.size, C.byref(rep)))
        return rep


class Plan:
    """A CUDA-graph launch of many windows over fixed device buffers."""

    def __init__(self, ctx: Context, rec: Records, offsets, window_ids, kernel_times: bool = False):
        self.ctx = ctx
        self.rec = rec
        off = np.ascontiguousarray(offsets, np.uint64)
        ids = np.ascontiguousarray(window_ids, np.uint64)
        h = C.c_void_p()
        ctx._c(lib().gnm_plan_create_ex(ctx.h, C.byref(rec.c), _ptr(off), _ptr(ids), ids.size,
                                        KERNEL_TIMES if kernel_times else 0, C.byref(h)))
        self.h = h

    def launch(self, stream=None):
        self.ctx._c(lib().gnm_plan_launch(self.h, _stream_ptr(stream)))

    def kernel_times(self):
        """[(kernel name, ms)] of the last launch, in launch order (plans made with kernel_times)."""
        ms = np.zeros(8, np.float32)
        kind = np.zeros(8, np.int32)
        n = C.c_size_t()
        self.ctx._c(lib().gnm_plan_kernel_times(self.h, _ptr(ms), _ptr(kind), 8, C.byref(n)))
        return [(KERNEL_NAMES[int(kind[i])], float(ms[i])) for i in range(n.value)]

    def close(self):
        if getattr(self, "h", None):
            lib().gnm_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Stream:
    """A streaming server over a context (gnm_stream_*): batches are admitted under a
    device-memory budget and processed on several CUDA streams as they arrive."""

    def __init__(self, ctx: Context, budget_bytes: int = 4 << 30, n_cuda_streams: int = 4,
                 max_queued: int = 65536, max_batch_records: int = 1 << 20):
        self.ctx = ctx
        c = StreamConfig()
        lib().gnm_stream_config_default(C.byref(c))
        c.budget_bytes = budget_bytes
        c.n_cuda_streams = n_cuda_streams
        c.max_queued = max_queued
        c.max_batch_records = max_batch_records
        h = C.c_void_p()
        ctx._c(lib().gnm_stream_open(ctx.h, C.byref(c), C.byref(h)))
        self.h = h
        self._held: Dict[int, list] = {}  # host batches kept alive until their window is reported
        self._buf = (WindowDone * 1024)()

    def submit(self, rec: "Records", window_id: int, close: bool = False):
        self.ctx._c(lib().gnm_stream_submit(self.h, C.byref(rec.c), window_id, 1 if close else 0))
        self._held.setdefault(window_id, []).append(rec)

    def close_window(self, window_id: int):
        """Closes a window with no further records."""
        empty = RecordsC()
        self.ctx._c(lib().gnm_stream_submit(self.h, C.byref(empty), window_id, 1))

    def submit_many(self, pool: "Records", begin, count, window_ids, close=None) -> int:
        """Batches that are slices [begin[i], begin[i] + count[i]) of one pool, for window_ids[i]
        (closing it when close[i]); returns how many were taken (all, unless an error is raised)."""
        b = np.ascontiguousarray(begin, np.uint64)
        c = np.ascontiguousarray(count, np.uint64)
        w = np.ascontiguousarray(window_ids, np.uint64)
        f = None if close is None else np.ascontiguousarray(close, np.uint8)
        n = C.c_size_t()
        st = lib().gnm_stream_submit_many(self.h, C.byref(pool.c), _ptr(b), _ptr(c), _ptr(w), _ptr(f), b.size,
                                          C.byref(n))
        for wid in np.unique(w[:n.value]):
            self._held.setdefault(int(wid), []).append(pool)
        self.ctx._c(st)
        return n.value

    def poll(self, wait_all: bool = False, queued: bool = False):
        """Windows completed since the last poll: list of (window_id, records, latency_ms, status)
        (with queued=True a fifth item: queued_ms)."""
        out = []
        wait = 1 if wait_all else 0
        while True:
            n = C.c_size_t()
            self.ctx._c(lib().gnm_stream_poll(self.h, self._buf, len(self._buf), C.byref(n), wait))
            for i in range(n.value):
                d = self._buf[i]
                r = (int(d.window_id), int(d.records), float(d.latency_ms), int(d.status))
                out.append(r + (float(d.queued_ms),) if queued else r)
                self._held.pop(int(d.window_id), None)
            if n.value < len(self._buf):
                return out
            wait = 0

    def stats(self) -> Dict[str, float]:
        st = StreamStats()
        self.ctx._c(lib().gnm_stream_stats_get(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in StreamStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().gnm_stream_close(self.h)
            self.h = None
            self._held.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
