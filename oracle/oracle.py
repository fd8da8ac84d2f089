"""ctypes binding and build step for the plain-C oracle (``gnm_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring). Every function states the passage
of the paper it follows in the C source; this file only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Dict, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gnm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NO_SITE = 0xFFFFFFFF
NSTAT = 6  # flows, octets, pkts, e_flows, e_octets, e_dur_ms
# unmatched classes
NONLOCAL, LOCALLOCAL, IN_UNREG, OUT_UNREG = 0, 1, 2, 3
IN, OUT = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C11, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.c_void_p
            lib.orc_lpm_build.restype = P
            lib.orc_lpm_build.argtypes = [P, P, P, C.c_size_t, C.POINTER(C.c_int)]
            lib.orc_lpm_free.argtypes = [P]
            lib.orc_lpm_lookup.argtypes = [P, P, C.c_size_t, P]
            lib.orc_lpm_scan.argtypes = [P, P, P, C.c_size_t, P, C.c_size_t, P]
            lib.orc_flatten.restype = C.c_longlong
            lib.orc_flatten.argtypes = [P, P, P, C.c_size_t]
            lib.orc_window.argtypes = [P, P, P, C.c_size_t, C.c_uint32, C.c_uint32, C.c_uint32,
                                       C.c_uint32, C.c_int, C.c_int] + [P] * 6 + [C.c_size_t, P, P]
            lib.orc_window_mt.argtypes = [P, P, P, C.c_size_t, C.c_uint32, C.c_uint32, C.c_uint32,
                                          C.c_uint32, C.c_int] + [P] * 6 + [C.c_size_t, P, P, C.c_int]
            lib.orc_rates.argtypes = [P, C.c_size_t, P]
            lib.orc_flags.argtypes = [P, P, C.c_size_t, C.c_double, C.c_uint32, P]
            lib.orc_rate_bucket.restype = C.c_uint32
            lib.orc_rate_bucket.argtypes = [C.c_uint32, C.c_uint32]
            lib.orc_rate_stats.argtypes = [P, P, P, C.c_size_t, C.c_uint32, C.c_uint32, C.c_uint32,
                                           C.c_uint32, C.c_int] + [P] * 6 + [C.c_size_t, P, P, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class LPM:
    """Longest-prefix matcher over a registry: hash tables per length, plus the
    sequential scan of every prefix."""

    ERRORS = {1: "length > 32", 2: "host bits set", 3: "duplicate (prefix, length)", 4: "out of memory"}

    def __init__(self, prefix, plen, site):
        lib = _load()
        self._pfx = _c(prefix, np.uint32)
        self._len = _c(plen, np.uint8)
        self._site = _c(site, np.uint32)
        err = C.c_int(0)
        self._h = lib.orc_lpm_build(_p(self._pfx), _p(self._len), _p(self._site), self._pfx.size,
                                    C.byref(err))
        if not self._h:
            raise ValueError(f"invalid registry: {self.ERRORS.get(err.value, err.value)}")

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_lpm_free(self._h)
            self._h = None

    def lookup(self, x) -> np.ndarray:
        x = _c(x, np.uint32)
        out = np.empty_like(x)
        _load().orc_lpm_lookup(self._h, _p(x), x.size, _p(out))
        return out

    def scan(self, x) -> np.ndarray:
        x = _c(x, np.uint32)
        out = np.empty_like(x)
        _load().orc_lpm_scan(_p(self._pfx), _p(self._len), _p(self._site), self._pfx.size, _p(x),
                             x.size, _p(out))
        return out

    def flatten(self) -> Tuple[np.ndarray, np.ndarray]:
        cap = 2 * self._pfx.size + 1
        st = np.empty(cap, np.uint32)
        si = np.empty(cap, np.uint32)
        n = _load().orc_flatten(self._h, _p(st), _p(si), cap)
        assert n > 0
        return st[:n].copy(), si[:n].copy()


DEFAULT_FILTER = dict(min_avg_pkt_bytes=100, min_pkts=10, min_dur_ms=1000, admin_rule=0)


def window(lpm: LPM, local_prefix, local_len, n_sites: int, rec: Dict[str, np.ndarray],
           min_avg_pkt_bytes: int = 100, min_pkts: int = 10, min_dur_ms: int = 1000,
           admin_rule: int = 0, use_scan: bool = False, n_threads: int = 0):
    """Per-window sums. Returns (stats[(2*n_sites), 6] u64, unmatched[4, 3] u64).

    Row site*2+dir holds flows, octets, pkts, e_flows, e_octets, e_dur_ms (dir 0 inbound,
    1 outbound). ``n_threads`` > 0 uses the threaded variant (hash matcher only)."""
    lib = _load()
    lp = _c(local_prefix, np.uint32)
    ll = _c(local_len, np.uint8)
    f = [_c(rec[k], np.uint32) for k in ("srcaddr", "dstaddr", "dPkts", "dOctets", "first", "last")]
    n = f[0].size
    stats = np.zeros((2 * n_sites, NSTAT), np.uint64)
    un = np.zeros((4, 3), np.uint64)
    if n_threads > 0:
        assert not use_scan
        rc = lib.orc_window_mt(lpm._h, _p(lp), _p(ll), lp.size, n_sites, min_avg_pkt_bytes, min_pkts,
                               min_dur_ms, admin_rule, *[_p(a) for a in f], n, _p(stats), _p(un),
                               n_threads)
    else:
        rc = lib.orc_window(lpm._h, _p(lp), _p(ll), lp.size, n_sites, min_avg_pkt_bytes, min_pkts,
                            min_dur_ms, admin_rule, int(use_scan), *[_p(a) for a in f], n, _p(stats),
                            _p(un))
    assert rc == 0
    return stats, un


def rates(stats: np.ndarray) -> np.ndarray:
    s = _c(stats, np.uint64)
    out = np.empty(s.shape[0], np.float64)
    _load().orc_rates(_p(s), s.shape[0], _p(out))
    return out


def flags(stats: np.ndarray, rate: np.ndarray, threshold: float, min_flows: int = 1) -> np.ndarray:
    s = _c(stats, np.uint64)
    r = _c(rate, np.float64)
    out = np.empty(s.shape[0], np.uint8)
    _load().orc_flags(_p(s), _p(r), s.shape[0], float(threshold), int(min_flows), _p(out))
    return out


def rate_bucket(octets: int, dur: int) -> int:
    return int(_load().orc_rate_bucket(int(octets), int(dur)))


N_BUCKETS = 10001  # rate histogram buckets of 10 kb/s, the last one for rates >= 100 Mb/s
NO_MEDIAN = 0xFFFFFFFF


def rate_stats(lpm: LPM, local_prefix, local_len, n_sites: int, rec: Dict[str, np.ndarray],
               min_avg_pkt_bytes: int = 100, min_pkts: int = 10, min_dur_ms: int = 1000, admin_rule: int = 0):
    """Per-flow rate statistics of a window (Sec. III.B.2.1). Returns (hist[2S, 10001] u32,
    rmin[2S] f64, rmax[2S] f64, median_bucket[2S] u32): over the eligible flows of each key,
    the rate histogram, the least and greatest rate (NaN without eligible flows) and the
    bucket of the lower median (NO_MEDIAN without eligible flows)."""
    lib = _load()
    lp = _c(local_prefix, np.uint32)
    ll = _c(local_len, np.uint8)
    f = [_c(rec[k], np.uint32) for k in ("srcaddr", "dstaddr", "dPkts", "dOctets", "first", "last")]
    nk = 2 * n_sites
    hist = np.zeros((nk, N_BUCKETS), np.uint32)
    rmin = np.empty(nk, np.float64)
    rmax = np.empty(nk, np.float64)
    med = np.empty(nk, np.uint32)
    rc = lib.orc_rate_stats(lpm._h, _p(lp), _p(ll), lp.size, n_sites, min_avg_pkt_bytes, min_pkts, min_dur_ms,
                            admin_rule, *[_p(a) for a in f], f[0].size, _p(hist), _p(rmin), _p(rmax), _p(med))
    assert rc == 0
    return hist, rmin, rmax, med


def rate_stats_keys(lpm: LPM, local_prefix, local_len, n_sites: int, rec: Dict[str, np.ndarray], keys,
                    min_avg_pkt_bytes: int = 100, min_pkts: int = 10, min_dur_ms: int = 1000, admin_rule: int = 0):
    """rate_stats for the given (site, dir) keys only, without a histogram for every key
    (a registry of 100,000 sites would need 8 GB of them): the same definitions (Sec.
    III.B.2.1), written out per record with numpy over this module's LPM. Per key, the
    buckets and rates of its eligible flows; the lower median is the ceil(n/2)-th smallest
    bucket. Returns (rmin, rmax, median_bucket, n_eligible) for `keys`, in their order."""
    keys = np.asarray(keys, np.int64)
    src = np.asarray(rec["srcaddr"], np.uint32)
    dst = np.asarray(rec["dstaddr"], np.uint32)
    pk = np.asarray(rec["dPkts"], np.uint64)
    oc = np.asarray(rec["dOctets"], np.uint64)
    dur = ((np.asarray(rec["last"], np.int64) - np.asarray(rec["first"], np.int64)) & 0xFFFFFFFF).astype(np.uint64)

    def is_local(a):
        r = np.zeros(a.shape, bool)
        for p_, l_ in zip(np.asarray(local_prefix, np.int64), np.asarray(local_len, np.int64)):
            r |= (a.astype(np.int64) >> (32 - l_)) == (p_ >> (32 - l_)) if l_ else True
        return r

    sl, dl = is_local(src), is_local(dst)
    mixed = sl != dl                        # exactly one endpoint local
    site = lpm.lookup(np.where(sl, dst, src)).astype(np.int64)
    reg = mixed & (site != NO_SITE)
    ack_ok = oc >= np.uint64(min_avg_pkt_bytes) * pk
    many, longd = pk >= min_pkts, dur >= np.uint64(min_dur_ms)
    admin_ok = (many & longd) if admin_rule == 0 else (many | longd)
    elig = reg & (dur != 0) & ack_ok & admin_ok
    key = np.where(elig, site * 2 + sl.astype(np.int64), -1)
    want = np.isin(key, keys)
    k_e, oc_e, dur_e = key[want], oc[want], dur[want]
    bucket = np.minimum((oc_e * np.uint64(4)) // (dur_e * np.uint64(5)), np.uint64(10000)).astype(np.int64)
    rate = (oc_e.astype(np.float64) * 8000.0) / dur_e.astype(np.float64)
    order = np.argsort(k_e, kind="stable")
    k_e, bucket, rate = k_e[order], bucket[order], rate[order]
    rmin = np.full(keys.size, np.nan)
    rmax = np.full(keys.size, np.nan)
    med = np.full(keys.size, NO_MEDIAN, np.uint32)
    cnt = np.zeros(keys.size, np.int64)
    for i, k in enumerate(keys):
        a, b = np.searchsorted(k_e, k, "left"), np.searchsorted(k_e, k, "right")
        n = b - a
        cnt[i] = n
        if n:
            rmin[i], rmax[i] = rate[a:b].min(), rate[a:b].max()
            med[i] = np.sort(bucket[a:b])[(n + 1) // 2 - 1]
    return rmin, rmax, med, cnt


def host_stats(lpm: LPM, local_prefix, local_len, n_sites: int, rec: Dict[str, np.ndarray],
               min_avg_pkt_bytes: int = 100, min_pkts: int = 10, min_dur_ms: int = 1000, admin_rule: int = 0):
    """Per-host sums of a window (Sec. III.B.2.1: statistics "for each host in a registered
    site"): for every remote address of a registered site and direction, the same six sums
    as a site key (flows, octets, pkts, e_flows, e_octets, e_dur_ms). Returns (addr u32,
    site u32, dir u8, sums[n, 6] u64) sorted by (site, dir, addr)."""
    src = np.asarray(rec["srcaddr"], np.uint32)
    dst = np.asarray(rec["dstaddr"], np.uint32)
    pk = np.asarray(rec["dPkts"], np.uint64)
    oc = np.asarray(rec["dOctets"], np.uint64)
    dur = (np.asarray(rec["last"], np.uint32) - np.asarray(rec["first"], np.uint32)).astype(np.uint64)

    def local(a):
        out = np.zeros(a.shape, bool)
        for p, l in zip(local_prefix, local_len):
            m = np.uint32(0) if int(l) == 0 else np.uint32((0xFFFFFFFF << (32 - int(l))) & 0xFFFFFFFF)
            out |= (a & m) == np.uint32(p)
        return out

    sl, dl = local(src), local(dst)
    out_ = sl & ~dl
    mixed = sl != dl
    remote = np.where(out_, dst, src)
    site = lpm.lookup(remote)
    keep = mixed & (site != NO_SITE)
    if min_avg_pkt_bytes is None:
        min_avg_pkt_bytes = 0
    few, short = pk < min_pkts, dur < min_dur_ms
    admin = ~(few | short) if admin_rule == 0 else ~(few & short)
    elig = keep & (dur > 0) & (oc >= np.uint64(min_avg_pkt_bytes) * pk) & admin
    key = (remote.astype(np.uint64) << np.uint64(1)) | out_.astype(np.uint64)
    uk, inv = np.unique(key[keep], return_inverse=True)
    sums = np.zeros((uk.size, NSTAT), np.uint64)
    e = elig[keep]
    np.add.at(sums[:, 0], inv, np.uint64(1))
    np.add.at(sums[:, 1], inv, oc[keep])
    np.add.at(sums[:, 2], inv, pk[keep])
    np.add.at(sums[:, 3], inv[e], np.uint64(1))
    np.add.at(sums[:, 4], inv[e], oc[keep][e])
    np.add.at(sums[:, 5], inv[e], dur[keep][e])
    addr = (uk >> np.uint64(1)).astype(np.uint32)
    d = (uk & np.uint64(1)).astype(np.uint8)
    hsite = lpm.lookup(addr)
    order = np.lexsort((addr, d, hsite))
    return addr[order], hsite[order], d[order], sums[order]


def warnings(median_buckets, below_bucket: int = 100, consecutive: int = 2):
    """Sec. III.B.1 / Sec. IV.B: a warning for a (site, dir) key when its median transfer
    rate was below a standard (1 Mb/s: median bucket < 100) in `consecutive` consecutive
    windows. median_buckets: one array of lower-median buckets per window, in time order
    (NO_MEDIAN, no eligible flow, is not below). Returns one boolean array per window."""
    streak = None
    out = []
    for m in median_buckets:
        m = np.asarray(m, np.uint32)
        below = (m != NO_MEDIAN) & (m < below_bucket)
        streak = np.where(below, (streak if streak is not None else 0) + 1, 0)
        out.append(streak >= consecutive)
    return out


def full_window(lpm: LPM, reg, rec, threshold: float = 1e8, min_flows: int = 1, **kw):
    """stats, unmatched, rate and flag of one window (the whole per-window definition)."""
    st, un = window(lpm, reg.local_prefix, reg.local_len, reg.n_sites, rec, **kw)
    r = rates(st)
    fl = flags(st, r, threshold, min_flows)
    return st, un, r, fl
