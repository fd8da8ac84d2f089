"""Seeded synthetic inputs shaped like NetFlow v5 flow windows and site registries.

This module only draws inputs: site registries (prefix, length, site id), local-site
prefixes and struct-of-arrays record batches. It computes nothing the analysis computes
(no prefix matching, no filtering, no sums, no rates); both the CPU oracle and the CUDA
library consume what it produces.

Record model (stated once, used by every workload):
  * remote endpoint: with probability ``p_reg`` a registered site drawn from a Zipf(s)
    popularity law, then one of that site's prefixes uniformly, then a uniform address
    inside the prefix; otherwise a uniform address inside one of the reserved
    "unregistered" blocks that no registry prefix may overlap;
  * local endpoint: uniform inside one of the local prefixes;
  * direction: inbound (remote is the source) with probability ``p_in``;
  * dOctets = clamp(round(exp(N(mu, sigma))), 1, 2^32-1);
  * average packet size: 75% U[576, 1500] bytes (data), 25% U[40, 64] (ACK-like),
    dPkts = clamp(ceil(dOctets / avg), 1, 2^32-1);
  * duration U[1, 60000] ms, First = t0 + U[0, 60000), Last = First + duration (mod 2^32);
  * ports uniform 16-bit, protocol 6 with probability 0.9 else 17 (never read).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np

U32 = np.uint32
MAX_U32 = (1 << 32) - 1


@dataclasses.dataclass
class Registry:
    prefix: np.ndarray        # uint32, host bits zero
    plen: np.ndarray          # uint8, 0..32
    site: np.ndarray          # uint32, dense ids in [0, n_sites)
    n_sites: int
    local_prefix: np.ndarray  # uint32
    local_len: np.ndarray     # uint8
    holes: np.ndarray         # int64 [k, 2] half-open blocks never registered
    nested: np.ndarray        # bool per prefix: placed inside a shorter prefix

    @property
    def n(self) -> int:
        return int(self.prefix.shape[0])


def _size(plen: np.ndarray) -> np.ndarray:
    return np.left_shift(np.int64(1), (32 - plen.astype(np.int64)))


def _free_of(cs: np.ndarray, ce: np.ndarray, occ_s: np.ndarray, occ_e: np.ndarray) -> np.ndarray:
    """True where [cs, ce) overlaps none of the sorted disjoint blocks [occ_s, occ_e)."""
    if occ_s.size == 0:
        return np.ones(cs.shape, dtype=bool)
    i = np.searchsorted(occ_s, cs, side="right") - 1
    ok = np.ones(cs.shape, dtype=bool)
    has_prev = i >= 0
    ok[has_prev] &= occ_e[i[has_prev]] <= cs[has_prev]
    j = i + 1
    has_next = j < occ_s.size
    ok[has_next] &= occ_s[j[has_next]] >= ce[has_next]
    return ok


def _self_disjoint(cs: np.ndarray, ce: np.ndarray) -> np.ndarray:
    """Greedy mask keeping candidates (in start order) that overlap no earlier one."""
    order = np.argsort(cs, kind="stable")
    s, e = cs[order], ce[order]
    prev_max = np.maximum.accumulate(np.concatenate([[-1], e[:-1]]))
    keep_sorted = s >= prev_max
    keep = np.zeros(cs.shape, dtype=bool)
    keep[order] = keep_sorted
    return keep


def _insert(occ_s, occ_e, s, e):
    cs = np.concatenate([occ_s, s])
    ce = np.concatenate([occ_e, e])
    o = np.argsort(cs, kind="stable")
    return cs[o], ce[o]


def _place(rng, lens: np.ndarray, occ_s: np.ndarray, occ_e: np.ndarray, lo: int = 0,
           hi: int = 1 << 32, max_rounds: int = 200):
    """Place aligned prefixes of the given lengths at random without overlapping the
    occupied blocks or each other (rejection sampling in vectorised rounds)."""
    starts = np.full(lens.shape, -1, dtype=np.int64)
    todo = np.arange(lens.size)
    for _ in range(max_rounds):
        if todo.size == 0:
            break
        ln = lens[todo].astype(np.int64)
        size = _size(ln)
        nslots = np.maximum((hi - lo) // size, 1)
        slot = (rng.random(todo.size) * nslots).astype(np.int64)
        cs = lo + slot * size
        ce = cs + size
        ok = _free_of(cs, ce, occ_s, occ_e) & (ce <= hi)
        ok &= _self_disjoint(np.where(ok, cs, -1 - np.arange(todo.size)), np.where(ok, ce, -np.arange(todo.size)))
        good = todo[ok]
        starts[good] = cs[ok]
        occ_s, occ_e = _insert(occ_s, occ_e, cs[ok], ce[ok])
        todo = todo[~ok]
    if todo.size:
        raise RuntimeError(f"could not place {todo.size} prefixes")
    return starts, occ_s, occ_e


def length_weights_peaked(lo: int, hi: int, peak: int, up: float = 0.6, down: float = 0.5) -> Dict[int, float]:
    """Relative frequency per prefix length: rises as 2^(up*(l-peak)) up to ``peak``
    and falls as 2^(-down*(l-peak)) beyond it (many long prefixes, few short ones,
    so the registry stays placeable without overlap)."""
    w = {}
    for l in range(lo, hi + 1):
        w[l] = 2.0 ** (up * (l - peak)) if l <= peak else 2.0 ** (-down * (l - peak))
    return w


def make_registry(n_sites: int, n_prefixes: int, len_weights: Dict[int, float],
                  nest_frac: float, seed: int, n_local: int = 2, local_len: int = 16,
                  n_holes: int = 8, hole_len: int = 12, max_nested_len: int = 30) -> Registry:
    """Registry of ``n_prefixes`` prefixes for ``n_sites`` sites.

    ``1 - nest_frac`` of the prefixes are mutually disjoint; the rest are placed inside
    a shorter prefix of another site (depth one), so that longest-prefix match is
    needed. Local prefixes and the reserved unregistered blocks overlap nothing.
    """
    rng = np.random.default_rng(seed)
    occ_s = np.zeros(0, np.int64)
    occ_e = np.zeros(0, np.int64)
    # local /16s and unregistered holes first (kept out of 0/8 and 224/3 for realism)
    lo_space, hi_space = 1 << 24, 224 << 24
    local_lens = np.full(n_local, local_len, np.int64)
    local_s, occ_s, occ_e = _place(rng, local_lens, occ_s, occ_e, lo_space, hi_space)
    hole_lens = np.full(n_holes, hole_len, np.int64)
    hole_s, occ_s, occ_e = _place(rng, hole_lens, occ_s, occ_e, lo_space, hi_space)

    n_nested = int(round(nest_frac * n_prefixes))
    n_top = n_prefixes - n_nested
    ls = np.array(sorted(len_weights), dtype=np.int64)
    w = np.array([len_weights[l] for l in ls], dtype=np.float64)
    top_lens = rng.choice(ls, size=n_top, p=w / w.sum())
    top_lens = np.sort(top_lens)  # shortest first: hardest to place
    top_s = np.empty(n_top, np.int64)
    # place shortest lengths first, length by length
    for l in np.unique(top_lens):
        idx = np.nonzero(top_lens == l)[0]
        s, occ_s, occ_e = _place(rng, top_lens[idx], occ_s, occ_e, lo_space, hi_space)
        top_s[idx] = s
    # sites of top-level prefixes: every site gets at least one, rest uniform
    top_site = rng.integers(0, n_sites, size=n_top, dtype=np.int64)
    k = min(n_sites, n_top)
    top_site[rng.permutation(n_top)[:k]] = rng.permutation(n_sites)[:k]

    nest_s = np.zeros(0, np.int64)
    nest_l = np.zeros(0, np.int64)
    nest_site = np.zeros(0, np.int64)
    if n_nested:
        L = max_nested_len
        parent_ok = np.nonzero(top_lens <= L - 1)[0]
        par = parent_ok[rng.integers(0, parent_ok.size, size=n_nested)]
        pl = top_lens[par]
        cl = pl + 1 + (rng.random(n_nested) * (L - pl)).astype(np.int64)
        cl = np.minimum(cl, L)
        nest_s = np.full(n_nested, -1, np.int64)
        todo = np.arange(n_nested)
        occ_cs = np.zeros(0, np.int64)
        occ_ce = np.zeros(0, np.int64)
        for rnd in range(400):
            if todo.size == 0:
                break
            if rnd % 10 == 9:  # a crowded parent: draw another parent and length
                par[todo] = parent_ok[rng.integers(0, parent_ok.size, size=todo.size)]
                pl[todo] = top_lens[par[todo]]
                cl[todo] = np.minimum(pl[todo] + 1 + (rng.random(todo.size) * (L - pl[todo])).astype(np.int64), L)
            size = _size(cl[todo])
            psize = _size(pl[todo])
            slot = (rng.random(todo.size) * (psize // size)).astype(np.int64)
            cs = top_s[par[todo]] + slot * size
            ce = cs + size
            ok = _free_of(cs, ce, occ_cs, occ_ce)
            ok &= _self_disjoint(np.where(ok, cs, -1 - np.arange(todo.size)), np.where(ok, ce, -np.arange(todo.size)))
            nest_s[todo[ok]] = cs[ok]
            occ_cs, occ_ce = _insert(occ_cs, occ_ce, cs[ok], ce[ok])
            todo = todo[~ok]
        keep = nest_s >= 0
        nest_s, nest_l, par = nest_s[keep], cl[keep], par[keep]
        # a nested prefix belongs to a different site than its parent
        off = rng.integers(1, max(n_sites, 2), size=nest_s.size)
        nest_site = (top_site[par] + off) % n_sites

    prefix = np.concatenate([top_s, nest_s]).astype(np.uint32)
    plen = np.concatenate([top_lens, nest_l]).astype(np.uint8)
    site = np.concatenate([top_site, nest_site]).astype(np.uint32)
    nested = np.concatenate([np.zeros(n_top, bool), np.ones(nest_s.size, bool)])
    perm = rng.permutation(prefix.size)
    holes = np.stack([hole_s, hole_s + (1 << (32 - hole_len))], axis=1)
    return Registry(prefix=prefix[perm], plen=plen[perm], site=site[perm], n_sites=n_sites,
                    local_prefix=local_s.astype(np.uint32), local_len=local_lens.astype(np.uint8),
                    holes=holes, nested=nested[perm])


def zipf_probs(n: int, s: float) -> np.ndarray:
    k = np.arange(1, n + 1, dtype=np.float64)
    p = k ** (-s)
    return p / p.sum()


def make_records(reg: Registry, n: int, seed: int, p_reg: float = 0.85, zipf_s: float = 1.1,
                 p_in: float = 0.3, t0_ms: int = 0, mu: float = 12.0, sigma: float = 3.0,
                 window_ms: int = 60000, t0_per_record: Optional[np.ndarray] = None,
                 with_remote: bool = False) -> Dict[str, np.ndarray]:
    """One struct-of-arrays batch of ``n`` records (see the module docstring). With
    ``with_remote`` the batch also carries "remote": the endpoint drawn as the remote one
    (registered or unregistered), i.e. the address each record's site lookup receives."""
    rng = np.random.default_rng(seed)
    # remote endpoint
    is_reg = rng.random(n) < p_reg
    n_reg = int(is_reg.sum())
    remote = np.empty(n, np.int64)
    # per-site prefix lists (CSR)
    order = np.argsort(reg.site, kind="stable")
    counts = np.bincount(reg.site, minlength=reg.n_sites)
    offs = np.concatenate([[0], np.cumsum(counts)])
    has = np.nonzero(counts > 0)[0]
    pop = zipf_probs(has.size, zipf_s)
    rank_to_site = has[rng.permutation(has.size)]
    cdf = np.cumsum(pop)
    cdf[-1] = 1.0
    rank = np.searchsorted(cdf, rng.random(n_reg), side="right")
    site = rank_to_site[np.minimum(rank, has.size - 1)]
    j = (rng.random(n_reg) * counts[site]).astype(np.int64)
    pidx = order[offs[site] + j]
    size = _size(reg.plen[pidx])
    remote[is_reg] = reg.prefix[pidx].astype(np.int64) + (rng.random(n_reg) * size).astype(np.int64)
    # unregistered: uniform inside a reserved hole
    n_un = n - n_reg
    h = rng.integers(0, reg.holes.shape[0], size=n_un)
    hs, he = reg.holes[h, 0], reg.holes[h, 1]
    remote[~is_reg] = hs + (rng.random(n_un) * (he - hs)).astype(np.int64)
    # local endpoint
    li = rng.integers(0, reg.local_prefix.size, size=n)
    lsize = _size(reg.local_len[li])
    local = reg.local_prefix[li].astype(np.int64) + (rng.random(n) * lsize).astype(np.int64)
    inbound = rng.random(n) < p_in
    src = np.where(inbound, remote, local).astype(np.uint32)
    dst = np.where(inbound, local, remote).astype(np.uint32)
    # volumes
    oct_f = np.rint(np.exp(rng.normal(mu, sigma, size=n)))
    octets = np.clip(oct_f, 1, MAX_U32).astype(np.uint32)
    ack = rng.random(n) < 0.25
    avg = np.where(ack, rng.integers(40, 65, size=n), rng.integers(576, 1501, size=n)).astype(np.float64)
    pkts = np.clip(np.ceil(octets.astype(np.float64) / avg), 1, MAX_U32).astype(np.uint32)
    dur = rng.integers(1, window_ms + 1, size=n, dtype=np.int64)
    base = np.int64(t0_ms) if t0_per_record is None else t0_per_record.astype(np.int64)
    first = (base + rng.integers(0, window_ms, size=n, dtype=np.int64)) & MAX_U32
    last = (first + dur) & MAX_U32
    out = {
        "srcaddr": src, "dstaddr": dst, "dPkts": pkts, "dOctets": octets,
        "first": first.astype(np.uint32), "last": last.astype(np.uint32),
        "srcport": rng.integers(0, 1 << 16, size=n, dtype=np.int64).astype(np.uint16),
        "dstport": rng.integers(0, 1 << 16, size=n, dtype=np.int64).astype(np.uint16),
        "prot": np.where(rng.random(n) < 0.9, 6, 17).astype(np.uint8),
    }
    if with_remote:
        out["remote"] = remote.astype(np.uint32)
    return out


FIELDS = ("srcaddr", "dstaddr", "dPkts", "dOctets", "first", "last")


# ----------------------------------------------------------------------------------
# Workload presets (sizes, distributions and seeds of the five evaluated workloads)
# ----------------------------------------------------------------------------------

C1_LEN = {l: 1.0 for l in range(12, 29)}          # /12../28 uniform
C2_LEN = length_weights_peaked(8, 30, peak=24)     # /8../30, mostly /20-/26
C3_LEN = length_weights_peaked(16, 30, peak=26)    # /16../30 for a million prefixes


def registry_c1(seed: int = 0) -> Registry:
    """500 sites, 2,000 disjoint prefixes /12-/28, two local /16s."""
    return make_registry(500, 2000, C1_LEN, 0.0, seed)


def registry_c2(seed: int = 1) -> Registry:
    """5,000 sites, 40,000 prefixes /8-/30, 20% nested inside another site's prefix."""
    return make_registry(5000, 40000, C2_LEN, 0.2, seed)


C2_24_LEN = length_weights_peaked(8, 24, peak=24)  # /8../24: what a /24 subnet catalog can hold


def registry_c2_24(seed: int = 1) -> Registry:
    """5,000 sites, 40,000 prefixes /8-/24, 20% nested: the hour's registry shape limited to
    the prefix lengths a /24 subnet hash table can expand."""
    return make_registry(5000, 40000, C2_24_LEN, 0.2, seed, max_nested_len=24)


def registry_c3(seed: int = 2, n_prefixes: int = 1_000_000, n_sites: int = 100_000) -> Registry:
    """100,000 sites, 1,000,000 prefixes /16-/30, 30% nested."""
    return make_registry(n_sites, n_prefixes, C3_LEN, 0.3, seed)


def lookup_keys_c3(reg: Registry, n: int = 10_000_000, seed: int = 12) -> np.ndarray:
    """Training lookups of the learned index: the remote endpoints of ``n`` records of the
    learned-index workload's distribution (90% registered, Zipf 0.9)."""
    return make_records(reg, n, seed=seed, p_reg=0.9, zipf_s=0.9, with_remote=True)["remote"]


def window_records_c1(reg: Registry, n: int = 100_000, seed: int = 0):
    """One one-minute window: 85% registered, Zipf(1.1), 30% inbound."""
    return make_records(reg, n, seed, p_reg=0.85, zipf_s=1.1, p_in=0.3)


def hour_records_c2(reg: Registry, n: int = 10_000_000, n_windows: int = 60, seed: int = 1,
                    wrap_window: int = 30):
    """Sixty one-minute windows back to back; window ``wrap_window`` straddles the
    32-bit millisecond wrap. Returns (records, offsets[n_windows+1])."""
    counts = np.full(n_windows, n // n_windows, np.int64)
    counts[: n - counts.sum()] += 1
    offsets = np.concatenate([[0], np.cumsum(counts)])
    base = np.int64(MAX_U32 + 1 - 30_000 - wrap_window * 60000)
    t0 = np.repeat(base + np.arange(n_windows, dtype=np.int64) * 60000, counts)
    rec = make_records(reg, n, seed, p_reg=0.85, zipf_s=1.0, p_in=0.3, t0_per_record=t0)
    return rec, offsets


def uneven_windows_c4(n_windows: int = 256, seed: int = 3, lo: int = 10_000, hi: int = 2_000_000,
                      median: float = 2e5, sigma: float = 1.0) -> np.ndarray:
    """Window sizes for the batched workload: clamp(round(lognormal(ln median, sigma)))."""
    rng = np.random.default_rng(seed)
    c = np.clip(np.rint(np.exp(rng.normal(math.log(median), sigma, size=n_windows))), lo, hi)
    return c.astype(np.int64)


def batched_records_c4(reg: Registry, counts: np.ndarray, seed: int = 3):
    offsets = np.concatenate([[0], np.cumsum(counts)])
    t0 = np.repeat(np.arange(counts.size, dtype=np.int64) * 60000, counts)
    rec = make_records(reg, int(offsets[-1]), seed, p_reg=0.85, zipf_s=1.1, p_in=0.3,
                       t0_per_record=t0)
    return rec, offsets


def serving_schedule_c5(hours: float = 24.0, mean_rate: float = 1e6, seed: int = 4,
                        size_lo: int = 1000, size_hi: int = 500_000):
    """Poisson batch arrivals with a diurnal factor f(t) = 1 + 0.7 sin(2 pi t / 86400).

    Returns arrival times (s) and batch sizes; the record rate averages ``mean_rate``.
    Arrivals are drawn by thinning a homogeneous process at the peak rate.
    """
    rng = np.random.default_rng(seed)
    mean_size = 0.5 * (size_lo + size_hi)
    lam_max = mean_rate * 1.7 / mean_size
    horizon = hours * 3600.0
    n_cand = int(lam_max * horizon * 1.05) + 16
    t = np.cumsum(rng.exponential(1.0 / lam_max, size=n_cand))
    t = t[t < horizon]
    f = 1.0 + 0.7 * np.sin(2 * np.pi * t / 86400.0)
    keep = rng.random(t.size) < f / 1.7
    t = t[keep]
    sizes = rng.integers(size_lo, size_hi + 1, size=t.size)
    return t, sizes


def split_windows(rec: Dict[str, np.ndarray], offsets: Sequence[int]) -> List[Dict[str, np.ndarray]]:
    return [{k: v[offsets[i]:offsets[i + 1]] for k, v in rec.items()} for i in range(len(offsets) - 1)]
