"""Pins of the CPU oracle against facts that do not come from the oracle itself:
hand-worked cases, brute force, closed forms, invariants and library routines.

The paper prints no worked example (no record with its site, rate or bucket), so the
hand-worked window in tests/golden/window_hand.json carries the definitions of
Sec. III.B.1-III.B.2.1 and Sec. IV.B through values computed by hand.
"""
import ipaddress
import json
import os

import numpy as np
import pytest

import flowgen as fg
import oracle
from oracle import rmi_ref

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def ip(s):
    return int(ipaddress.IPv4Address(s))


def load_hand():
    with open(os.path.join(GOLD, "window_hand.json")) as f:
        g = json.load(f)
    reg = np.array([(ip(a), l, s) for a, l, s in g["registry"]], dtype=np.int64)
    loc = np.array([(ip(a), l) for a, l in g["local"]], dtype=np.int64)
    cols = {k: [] for k in fg.FIELDS}
    for r in g["records"]:
        cols["srcaddr"].append(ip(r[0]))
        cols["dstaddr"].append(ip(r[1]))
        cols["dPkts"].append(r[2])
        cols["dOctets"].append(r[3])
        cols["first"].append(r[4])
        cols["last"].append(r[5])
    rec = {k: np.array(v, dtype=np.uint32) for k, v in cols.items()}
    return g, reg, loc, rec


# ----------------------------------------------------------------- prefix match

HAND_REG = [("10.0.0.0", 8, 0), ("10.1.0.0", 16, 1), ("10.1.2.0", 24, 2), ("10.1.2.4", 30, 3),
            ("10.1.3.0", 24, 4), ("255.255.255.255", 32, 5), ("192.0.2.0", 25, 6),
            ("192.0.2.128", 25, 7)]
HAND_CASES = [("10.0.0.0", 0), ("9.255.255.255", oracle.NO_SITE), ("10.255.255.255", 0),
              ("11.0.0.0", oracle.NO_SITE), ("10.1.0.0", 1), ("10.1.1.255", 1), ("10.1.2.0", 2),
              ("10.1.2.3", 2), ("10.1.2.4", 3), ("10.1.2.7", 3), ("10.1.2.8", 2), ("10.1.2.255", 2),
              ("10.1.3.0", 4), ("10.1.3.255", 4), ("10.1.4.0", 1), ("10.2.0.0", 0),
              ("255.255.255.255", 5), ("255.255.255.254", oracle.NO_SITE), ("0.0.0.0", oracle.NO_SITE),
              ("192.0.2.127", 6), ("192.0.2.128", 7), ("192.0.3.0", oracle.NO_SITE)]


def _hand_lpm(extra=()):
    rows = HAND_REG + list(extra)
    p = np.array([ip(a) for a, _, _ in rows], np.uint32)
    l = np.array([b for _, b, _ in rows], np.uint8)
    s = np.array([c for _, _, c in rows], np.uint32)
    return oracle.LPM(p, l, s)


def test_lpm_hand_cases_hash_and_scan():
    m = _hand_lpm()
    x = np.array([ip(a) for a, _ in HAND_CASES], np.uint32)
    want = np.array([s for _, s in HAND_CASES], np.uint32)
    np.testing.assert_array_equal(m.lookup(x), want)
    np.testing.assert_array_equal(m.scan(x), want)


def test_lpm_default_route():
    m = _hand_lpm(extra=[("0.0.0.0", 0, 9)])
    x = np.array([ip(a) for a, _ in HAND_CASES], np.uint32)
    want = np.array([9 if s == oracle.NO_SITE else s for _, s in HAND_CASES], np.uint32)
    np.testing.assert_array_equal(m.lookup(x), want)
    np.testing.assert_array_equal(m.scan(x), want)


@pytest.mark.parametrize("seed", range(6))
def test_lpm_hash_equals_bruteforce_scan(seed):
    """Random nested registries inside one /16 (plus a few covering prefixes); every one
    of the 65,536 addresses of the /16 and its neighbours is matched both ways."""
    rng = np.random.default_rng(seed)
    base = ip("172.16.0.0")
    rows = {}
    for _ in range(60):
        l = int(rng.integers(16, 33))
        a = base + int(rng.integers(0, 1 << 16))
        a &= (0xFFFFFFFF << (32 - l)) & 0xFFFFFFFF
        rows[(a, l)] = int(rng.integers(0, 20))
    rows[(ip("172.0.0.0"), 8)] = 21
    rows[(ip("172.16.0.0"), 12)] = 22
    p = np.array([k[0] for k in rows], np.uint32)
    l = np.array([k[1] for k in rows], np.uint8)
    s = np.array(list(rows.values()), np.uint32)
    m = oracle.LPM(p, l, s)
    x = (np.arange(-256, (1 << 16) + 256, dtype=np.int64) + base).astype(np.uint32)
    np.testing.assert_array_equal(m.lookup(x), m.scan(x))


def test_lpm_rejects_invalid():
    with pytest.raises(ValueError, match="host bits"):
        oracle.LPM(np.array([ip("10.0.0.1")], np.uint32), np.array([24], np.uint8), np.array([0], np.uint32))
    with pytest.raises(ValueError, match="length"):
        oracle.LPM(np.array([0], np.uint32), np.array([33], np.uint8), np.array([0], np.uint32))
    with pytest.raises(ValueError, match="duplicate"):
        oracle.LPM(np.array([ip("10.0.0.0")] * 2, np.uint32), np.array([8, 8], np.uint8),
                   np.array([0, 1], np.uint32))


def test_flatten_matches_lpm_at_every_boundary():
    reg = fg.registry_c2()
    m = oracle.LPM(reg.prefix, reg.plen, reg.site)
    st, si = m.flatten()
    assert st[0] == 0 and np.all(np.diff(st.astype(np.int64)) > 0)
    assert np.all(si[1:] != si[:-1])  # neighbours merged
    probes = np.concatenate([st.astype(np.int64), st.astype(np.int64) - 1, st.astype(np.int64) + 1,
                             np.random.default_rng(0).integers(0, 1 << 32, 100000)])
    probes = np.unique(probes[(probes >= 0) & (probes < (1 << 32))]).astype(np.uint32)
    idx = np.searchsorted(st, probes, side="right") - 1
    np.testing.assert_array_equal(si[idx], m.lookup(probes))


# ----------------------------------------------------------------------- window

def _gold_window(g, reg, loc, rec, **kw):
    m = oracle.LPM(reg[:, 0], reg[:, 1], reg[:, 2])
    return oracle.window(m, loc[:, 0], loc[:, 1], g["n_sites"], rec, **kw)


@pytest.mark.parametrize("use_scan", [False, True])
def test_hand_window(use_scan):
    g, reg, loc, rec = load_hand()
    st, un = _gold_window(g, reg, loc, rec, use_scan=use_scan)
    want = np.zeros_like(st)
    for row in g["expected_rows"]:
        want[row[0] * 2 + row[1]] = row[2:]
    np.testing.assert_array_equal(st, want)
    np.testing.assert_array_equal(un, np.array(g["expected_unmatched"], np.uint64))
    r = oracle.rates(st)
    for key, v in g["expected_rates_bps"].items():
        s, d = map(int, key.split(","))
        assert r[s * 2 + d] == pytest.approx(v, rel=1e-15)
    nan_rows = [i for i in range(st.shape[0]) if st[i, 5] == 0]
    assert np.all(np.isnan(r[nan_rows]))
    for thr, rows in g["thresholds"].items():
        fl = oracle.flags(st, r, float(thr))
        want_fl = np.zeros(st.shape[0], np.uint8)
        for s, d in rows:
            want_fl[s * 2 + d] = 1
        np.testing.assert_array_equal(fl, want_fl)


def test_hand_window_and_rule():
    g, reg, loc, rec = load_hand()
    st, _ = _gold_window(g, reg, loc, rec, admin_rule=1)
    want = np.zeros_like(st)
    for row in g["expected_rows"]:
        want[row[0] * 2 + row[1]] = row[2:]
    for row in g["admin_rule_and"]["changed_rows"]:
        want[row[0] * 2 + row[1]] = row[2:]
    np.testing.assert_array_equal(st, want)
    r = oracle.rates(st)
    for key, v in g["admin_rule_and"]["rates_bps"].items():
        s, d = map(int, key.split(","))
        assert r[s * 2 + d] == pytest.approx(v, rel=1e-15)


def _one_record_stats(pk, oc, first, last, **kw):
    """A single outbound record to a one-prefix registry; returns its row."""
    m = oracle.LPM(np.array([ip("10.0.0.0")], np.uint32), np.array([8], np.uint8),
                   np.array([0], np.uint32))
    rec = {k: np.array([v], np.uint32) for k, v in zip(
        fg.FIELDS, [ip("131.225.0.1"), ip("10.0.0.1"), pk, oc, first, last])}
    st, _ = oracle.window(m, np.array([ip("131.225.0.0")]), np.array([16]), 1, rec, **kw)
    return st[1]


@pytest.mark.parametrize("pk,oc,first,last,eligible", [
    (10, 1000, 0, 1000, True),       # avg exactly 100 B, 10 pkts, 1000 ms
    (10, 999, 0, 1000, False),       # avg 99.9 B
    (9, 900, 0, 1000, False),        # 9 packets
    (10, 1000, 0, 999, False),       # 999 ms
    (10, 1000, 7, 7, False),         # zero duration
    (10, 1000, 0xFFFFFF00, 0x2E8, True),  # Last < First: 1000 ms across the wrap
    (10, 1000, 1000, 0, True),       # Last < First: modulo 2^32 a 4,294,966,296 ms flow
    (0, 0, 0, 5000, False),          # no packets at all
])
def test_filter_boundaries(pk, oc, first, last, eligible):
    row = _one_record_stats(pk, oc, first, last)
    dur = (last - first) & 0xFFFFFFFF
    assert row[0] == 1 and row[1] == oc and row[2] == pk
    assert tuple(row[3:]) == ((1, oc, dur) if eligible else (0, 0, 0))


def test_filter_thresholds_are_parameters():
    row = _one_record_stats(5, 5000, 0, 500, min_pkts=5, min_dur_ms=500, min_avg_pkt_bytes=1000)
    assert tuple(row[3:]) == (1, 5000, 500)
    row = _one_record_stats(5, 4999, 0, 500, min_pkts=5, min_dur_ms=500, min_avg_pkt_bytes=1000)
    assert tuple(row[3:]) == (0, 0, 0)


def test_rate_closed_form_and_threshold():
    # 125,000 bytes in 1,000 ms = 1,000,000 bits/s exactly
    st = np.zeros((3, oracle.NSTAT), np.uint64)
    st[0] = [1, 125000, 100, 1, 125000, 1000]
    st[1] = [3, 10, 1, 2, 1, 3]          # 8000/3 b/s, inexact in binary
    st[2] = [4, 10, 1, 0, 0, 0]          # no eligible flow
    r = oracle.rates(st)
    assert r[0] == 1e6
    assert r[1] == np.float64(8000.0) / np.float64(3.0)
    assert np.isnan(r[2])
    np.testing.assert_array_equal(oracle.flags(st, r, 1e6), [0, 1, 0])
    np.testing.assert_array_equal(oracle.flags(st, r, np.nextafter(1e6, 2e6)), [1, 1, 0])
    np.testing.assert_array_equal(oracle.flags(st, r, 1e7, min_flows=2), [0, 1, 0])


def test_rate_large_sums_round_once():
    # sums above 2^53 convert to double with one rounding, then multiply, then divide
    eo = (1 << 60) + 12345
    ed = 3
    st = np.array([[1, eo, 1, 1, eo, ed]], np.uint64)
    r = oracle.rates(st)[0]
    assert r == (np.float64(eo) * np.float64(8000.0)) / np.float64(ed)


def _c1_window(n=20000, seed=5):
    reg = fg.registry_c1()
    rec = fg.window_records_c1(reg, n=n, seed=seed)
    return reg, rec, oracle.LPM(reg.prefix, reg.plen, reg.site)


def test_window_conservation_and_bounds():
    reg, rec, m = _c1_window()
    st, un = oracle.window(m, reg.local_prefix, reg.local_len, reg.n_sites, rec)
    tot_flows = st[:, 0].sum() + un[:, 0].sum()
    tot_oct = st[:, 1].sum() + un[:, 1].sum()
    tot_pk = st[:, 2].sum() + un[:, 2].sum()
    assert tot_flows == rec["srcaddr"].size
    assert tot_oct == rec["dOctets"].astype(np.uint64).sum()
    assert tot_pk == rec["dPkts"].astype(np.uint64).sum()
    assert np.all(st[:, 3] <= st[:, 0]) and np.all(st[:, 4] <= st[:, 1])
    # generated records always have exactly one local endpoint
    assert un[0, 0] == 0 and un[1, 0] == 0
    # eligible durations are bounded by the window's maximum flow duration
    assert np.all(st[:, 5] <= st[:, 3] * 60000)
    assert np.all(st[:, 5] >= st[:, 3] * 1000)


def test_window_permutation_and_split_invariance():
    reg, rec, m = _c1_window()
    a, ua = oracle.window(m, reg.local_prefix, reg.local_len, reg.n_sites, rec)
    perm = np.random.default_rng(1).permutation(rec["srcaddr"].size)
    b, ub = oracle.window(m, reg.local_prefix, reg.local_len, reg.n_sites,
                          {k: v[perm] for k, v in rec.items()})
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(ua, ub)
    cut = 7777
    p1, q1 = oracle.window(m, reg.local_prefix, reg.local_len, reg.n_sites, {k: v[:cut] for k, v in rec.items()})
    p2, q2 = oracle.window(m, reg.local_prefix, reg.local_len, reg.n_sites, {k: v[cut:] for k, v in rec.items()})
    np.testing.assert_array_equal(a, p1 + p2)
    np.testing.assert_array_equal(ua, q1 + q2)


def test_window_scan_equals_hash_and_threads():
    reg, rec, m = _c1_window(n=4000)
    a, ua = oracle.window(m, reg.local_prefix, reg.local_len, reg.n_sites, rec)
    b, ub = oracle.window(m, reg.local_prefix, reg.local_len, reg.n_sites, rec, use_scan=True)
    c, uc = oracle.window(m, reg.local_prefix, reg.local_len, reg.n_sites, rec, n_threads=3)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a, c)
    np.testing.assert_array_equal(ua, ub)
    np.testing.assert_array_equal(ua, uc)


def test_window_direction_from_numpy_definition():
    """Independent numpy restatement of the direction and key assignment on C1 data:
    per-key flow counts must agree with the oracle."""
    reg, rec, m = _c1_window(n=20000)
    st, un = oracle.window(m, reg.local_prefix, reg.local_len, reg.n_sites, rec)
    src, dst = rec["srcaddr"].astype(np.int64), rec["dstaddr"].astype(np.int64)

    def local(a):
        out = np.zeros(a.shape, bool)
        for p, l in zip(reg.local_prefix, reg.local_len):
            out |= (a >> (32 - int(l))) == (int(p) >> (32 - int(l)))
        return out

    sl, dl = local(src), local(dst)
    out_ = sl & ~dl
    in_ = dl & ~sl
    flat_s, flat_site = m.flatten()
    remote = np.where(out_, dst, src).astype(np.uint32)
    site = flat_site[np.searchsorted(flat_s, remote, side="right") - 1]
    key = site.astype(np.int64) * 2 + out_.astype(np.int64)
    ok = (out_ | in_) & (site != oracle.NO_SITE)
    counts = np.bincount(key[ok], minlength=2 * reg.n_sites)
    np.testing.assert_array_equal(st[:, 0], counts)
    assert un[3, 0] == np.sum(out_ & (site == oracle.NO_SITE))
    assert un[2, 0] == np.sum(in_ & (site == oracle.NO_SITE))


def test_rate_bucket_closed_form():
    # 1,250 bytes in 1 s = 10,000 b/s: first byte of bucket 1
    assert oracle.rate_bucket(1250, 1000) == 1
    assert oracle.rate_bucket(1249, 1000) == 0
    assert oracle.rate_bucket(1_250_000, 1000) == 1000           # 10 Mb/s
    assert oracle.rate_bucket(12_500_000, 1000) == 10000         # 100 Mb/s: last bucket
    assert oracle.rate_bucket(0xFFFFFFFF, 1) == 10000            # capped


# ---------------------------------------------------------- learned-index maths

def test_rate_stats_hand_case():
    """Three eligible outbound flows to one site plus one that the filters drop: rates 1, 3
    and 2 Mb/s (buckets 100, 300, 200), min 1e6, max 3e6, lower median the 2nd smallest
    (2 Mb/s, bucket 200); the other key has none."""
    reg = np.array([[ip("10.0.0.0"), 8, 0]])
    m = oracle.LPM(reg[:, 0], reg[:, 1], reg[:, 2])
    loc = ip("131.225.0.0")
    # octets, dur: 125,000 B in 1 s = 1 Mb/s; 375,000 B in 1 s = 3 Mb/s; 500,000 B in 2 s = 2 Mb/s
    oc = np.array([125_000, 375_000, 500_000, 125_000], np.uint32)
    dur = np.array([1000, 1000, 2000, 10], np.uint32)  # the last lasts 10 ms: administrative
    rec = {"srcaddr": np.full(4, loc + 5, np.uint32), "dstaddr": np.full(4, ip("10.1.2.3"), np.uint32),
           "dPkts": np.full(4, 100, np.uint32), "dOctets": oc, "first": np.full(4, 7, np.uint32),
           "last": (7 + dur).astype(np.uint32)}
    hist, rmin, rmax, med = oracle.rate_stats(m, [loc], [16], 1, rec)
    want = np.zeros((2, oracle.N_BUCKETS), np.uint32)
    want[1, [100, 200, 300]] = 1
    np.testing.assert_array_equal(hist, want)
    assert rmin[1] == 1e6 and rmax[1] == 3e6 and med[1] == 200
    assert np.isnan(rmin[0]) and np.isnan(rmax[0]) and med[0] == oracle.NO_MEDIAN


def test_rate_stats_against_sorted_rates():
    """Independent numpy restatement on C1 data: per key, the eligible flows' rates sorted,
    their least, greatest and ceil(n/2)-th values and its bucket; the histogram from numpy's
    bincount; histogram totals equal the window's eligible-flow counts."""
    reg, rec, m = _c1_window(n=30000, seed=9)
    hist, rmin, rmax, med = oracle.rate_stats(m, reg.local_prefix, reg.local_len, reg.n_sites, rec)
    st, _ = oracle.window(m, reg.local_prefix, reg.local_len, reg.n_sites, rec)
    np.testing.assert_array_equal(hist.sum(axis=1), st[:, 3])
    src, dst = rec["srcaddr"].astype(np.int64), rec["dstaddr"].astype(np.int64)

    def local(a):
        out = np.zeros(a.shape, bool)
        for p, l in zip(reg.local_prefix, reg.local_len):
            out |= (a >> (32 - int(l))) == (int(p) >> (32 - int(l)))
        return out

    sl, dl = local(src), local(dst)
    flat_s, flat_site = m.flatten()
    remote = np.where(sl & ~dl, dst, src).astype(np.uint32)
    site = flat_site[np.searchsorted(flat_s, remote, side="right") - 1]
    o = rec["dOctets"].astype(np.int64)
    pk = rec["dPkts"].astype(np.int64)
    d = (rec["last"].astype(np.int64) - rec["first"].astype(np.int64)) % (1 << 32)
    elig = (sl != dl) & (site != oracle.NO_SITE) & (d > 0) & (o >= 100 * pk) & (pk >= 10) & (d >= 1000)
    key = site.astype(np.int64) * 2 + (sl & ~dl)
    rate = o * 8000.0 / np.where(d > 0, d, 1)
    bucket = np.minimum(10000, (4 * o) // (5 * np.where(d > 0, d, 1)))
    for k in range(2 * reg.n_sites):
        sel = elig & (key == k)
        if not sel.any():
            assert np.isnan(rmin[k]) and med[k] == oracle.NO_MEDIAN
            continue
        r = np.sort(rate[sel])
        b = np.sort(bucket[sel])
        assert rmin[k] == r[0] and rmax[k] == r[-1]
        assert med[k] == b[(sel.sum() + 1) // 2 - 1]
        np.testing.assert_array_equal(hist[k], np.bincount(bucket[sel], minlength=oracle.N_BUCKETS))


def test_host_stats_sum_to_site_rows_and_hand_case():
    """Per-host sums: on the 500-site workload they add up, host by host, to the C oracle's
    per-site rows; a hand case gives two hosts of one site."""
    reg, rec, m = _c1_window(n=40000, seed=12)
    addr, site, d, sums = oracle.host_stats(m, reg.local_prefix, reg.local_len, reg.n_sites, rec)
    st, _ = oracle.window(m, reg.local_prefix, reg.local_len, reg.n_sites, rec)
    per_key = np.zeros_like(st)
    np.add.at(per_key, site.astype(np.int64) * 2 + d, sums)
    np.testing.assert_array_equal(per_key, st)
    assert len(np.unique(addr.astype(np.uint64) * 2 + d)) == addr.size  # one row per (host, dir)
    regh = np.array([[ip("10.0.0.0"), 8, 3]])
    mh = oracle.LPM(regh[:, 0], regh[:, 1], regh[:, 2])
    loc = ip("131.225.0.0")
    a, b = ip("10.0.0.1"), ip("10.0.0.2")
    rec = {"srcaddr": np.array([loc + 1, loc + 2, b, loc + 1], np.uint32),
           "dstaddr": np.array([a, a, loc + 9, ip("11.0.0.1")], np.uint32),
           "dPkts": np.array([10, 20, 30, 40], np.uint32), "dOctets": np.array([2000, 3000, 5000, 7000], np.uint32),
           "first": np.zeros(4, np.uint32), "last": np.array([1000, 500, 4000, 1000], np.uint32)}
    addr, site, d, sums = oracle.host_stats(mh, [loc], [16], 4, rec)
    assert addr.tolist() == [b, a] and site.tolist() == [3, 3] and d.tolist() == [0, 1]
    np.testing.assert_array_equal(sums, [[1, 5000, 30, 1, 5000, 4000], [2, 5000, 30, 1, 2000, 1000]])


def test_warnings_hand_sequence():
    """Four keys over five windows (median buckets; 99 is below 1 Mb/s, 100 is not):
    key 0 below in windows 1-3, key 1 alternates, key 2 below then without flows then
    below, key 3 below in every window."""
    N = oracle.NO_MEDIAN
    seq = [[100, 5, 99, 0], [99, 100, 99, 0], [50, 7, N, 0], [0, 100, 99, 0], [100, 8, 99, 0]]
    got = [w.tolist() for w in oracle.warnings(seq)]
    assert got == [[False, False, False, False],
                   [False, False, True, True],
                   [True, False, False, True],
                   [True, False, False, True],
                   [False, False, True, True]]
    # three windows in a row
    got3 = [w.tolist() for w in oracle.warnings(seq, consecutive=3)]
    assert got3[2] == [False, False, False, True] and got3[3] == [True, False, False, True]


def test_lstsq_line_equals_polyfit():
    rng = np.random.default_rng(0)
    x = rng.random(5000) * 1e6
    y = 3.5 * x - 17 + rng.normal(0, 50, x.size)
    a, b = rmi_ref.lstsq_line(x, y)
    pa, pb = np.polyfit(x, y, 1)
    assert a == pytest.approx(pa, rel=1e-10)
    assert b == pytest.approx(pb, rel=1e-8, abs=1e-6)


def test_linear_grad_finite_difference():
    rng = np.random.default_rng(1)
    z = rng.normal(size=1000)
    y = 2 * z + 1 + rng.normal(size=1000)
    w, c, h = 0.3, -0.2, 1e-6
    _, gw, gc = rmi_ref.linear_grad(w, c, z, y)
    fw = (rmi_ref.linear_grad(w + h, c, z, y)[0] - rmi_ref.linear_grad(w - h, c, z, y)[0]) / (2 * h)
    fc = (rmi_ref.linear_grad(w, c + h, z, y)[0] - rmi_ref.linear_grad(w, c - h, z, y)[0]) / (2 * h)
    assert gw == pytest.approx(fw, rel=1e-6)
    assert gc == pytest.approx(fc, rel=1e-6)


def test_mlp_grad_finite_difference():
    rng = np.random.default_rng(2)
    H = 32
    p = {"w1": rng.normal(size=H), "b1": rng.normal(size=H) * 0.1, "w2": rng.normal(size=H),
         "b2": 0.05}
    xn = rng.random(2000)
    y = np.sqrt(xn) * 100
    _, g = rmi_ref.mlp_loss_grad(p, xn, y)
    h = 1e-6
    for name in ("w1", "b1", "w2"):
        for j in (0, 7, 31):
            q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
            q[name][j] += h
            lp = rmi_ref.mlp_loss_grad(q, xn, y)[0]
            q[name][j] -= 2 * h
            lm = rmi_ref.mlp_loss_grad(q, xn, y)[0]
            assert g[name][j] == pytest.approx((lp - lm) / (2 * h), rel=1e-4, abs=1e-6)
    lp = rmi_ref.mlp_loss_grad({**p, "b2": p["b2"] + h}, xn, y)[0]
    lm = rmi_ref.mlp_loss_grad({**p, "b2": p["b2"] - h}, xn, y)[0]
    assert g["b2"] == pytest.approx((lp - lm) / (2 * h), rel=1e-6)
    # forward agrees with the explicit formula
    out = rmi_ref.mlp_forward(p, xn[:3])
    want = [sum(p["w2"][j] * max(p["w1"][j] * v + p["b1"][j], 0) for j in range(H)) + p["b2"] for v in xn[:3]]
    np.testing.assert_allclose(out, want, rtol=1e-12)


def test_eps_endpoints_bound_holds_and_is_tight():
    """The per-leaf error bound from range endpoints against predictions at many
    sampled addresses (all range boundaries +-1 and random ones)."""
    reg = fg.registry_c1()
    m = oracle.LPM(reg.prefix, reg.plen, reg.site)
    st, _ = m.flatten()
    n, L = st.size, 64
    # a crude monotone model: root and leaves from least squares on the starts
    pos = np.arange(n, dtype=np.float64)
    ra, rb = rmi_ref.lstsq_line(st.astype(np.float64) / 2 ** 32, pos * L / n)
    ra = max(ra, 0.0)
    leaf_of_start = rmi_ref.root_linear(ra, rb, st, L)
    a = np.zeros(L)
    b = np.zeros(L)
    x0 = np.zeros(L, np.int64)
    for l in range(L):
        sel = leaf_of_start == l
        if sel.sum() >= 2:
            x0[l] = int(st[sel][0])
            al, bl = rmi_ref.lstsq_line(st[sel].astype(np.float64) - x0[l], pos[sel])
            a[l], b[l] = max(al, 0.0), bl
    elo, ehi = rmi_ref.eps_endpoints_linear(st, ra, rb, a, b, x0, L)
    s64 = st.astype(np.int64)
    lf = rmi_ref.leaf_first_addresses(ra, rb, L)
    probes = np.concatenate([s64, s64 - 1, s64 + 1, lf, lf - 1,
                             np.random.default_rng(0).integers(0, 1 << 32, 200000)])
    probes = np.unique(probes[(probes >= 0) & (probes < (1 << 32))])
    t = np.searchsorted(st, probes.astype(np.uint32), side="right") - 1
    leaf = rmi_ref.root_linear(ra, rb, probes.astype(np.uint32), L)
    p = rmi_ref.leaf_predict(a, b, x0, leaf, probes, n)
    assert np.all(p - t <= elo[leaf])
    assert np.all(t - p <= ehi[leaf])
    # tight: the bound is reached at some sampled endpoint of every non-empty leaf
    got_lo = np.zeros(L, np.int64)
    got_hi = np.zeros(L, np.int64)
    np.maximum.at(got_lo, leaf, np.maximum(p - t, 0))
    np.maximum.at(got_hi, leaf, np.maximum(t - p, 0))
    np.testing.assert_array_equal(got_lo, elo)
    np.testing.assert_array_equal(got_hi, ehi)


# ------------------------------------------------ learned index: hand-worked FP32 pins

def _f(s):
    return float.fromhex(s) if isinstance(s, str) and s not in ("nan", "inf", "-inf") else float(s)


def _rmi_hand():
    with open(os.path.join(GOLD, "rmi_hand.json")) as f:
        return json.load(f)


def test_rmi_hand_xnorm():
    """fl(fl(x) * 2^-32), with the FP32 rounding of x worked out by hand."""
    g = _rmi_hand()
    x = np.array([c["x"] for c in g["xnorm"]], np.uint32)
    want = np.array([_f(c["xn"]) for c in g["xnorm"]], np.float32)
    got = rmi_ref.xnorm(x)
    assert got.dtype == np.float32
    np.testing.assert_array_equal(got, want)


def test_rmi_hand_clamp_floor():
    g = _rmi_hand()["clamp_floor"]
    v = np.array([_f(s) for s in g["v"]], np.float32)
    np.testing.assert_array_equal(rmi_ref._clamp_floor(v, g["n"]), np.array(g["want"]))


def test_rmi_hand_root_linear():
    """Linear root by hand, including keys that FP32 rounding sends to the next leaf."""
    for blk in _rmi_hand()["root_linear"]:
        x = np.array([c["x"] for c in blk["cases"]], np.uint32)
        want = np.array([c["leaf"] for c in blk["cases"]])
        got = rmi_ref.root_linear(_f(blk["ra"]), _f(blk["rb"]), x, blk["L"])
        np.testing.assert_array_equal(got, want)


def test_rmi_hand_root_mlp():
    """1 -> 2 -> 1 ReLU root by hand (negative output clamped to 0, large output to L-1)."""
    for blk in _rmi_hand()["root_mlp"]:
        p = {"w1": np.array([_f(s) for s in blk["w1"]]), "b1": np.array([_f(s) for s in blk["b1"]]),
             "w2": np.array([_f(s) for s in blk["w2"]]), "b2": _f(blk["b2"])}
        x = np.array([c["x"] for c in blk["cases"]], np.uint32)
        want = np.array([c["leaf"] for c in blk["cases"]])
        np.testing.assert_array_equal(rmi_ref.root_mlp(p, x, blk["L"]), want)


def test_rmi_hand_leaf_first_addresses():
    """First address of every leaf of a monotone linear root: powers of two where FP32 is
    exact, and the rounding ties at 2^29, 1.5*2^30 and 2.5*2^30 worked out by hand."""
    for blk in _rmi_hand()["leaf_first_addresses"]:
        got = rmi_ref.leaf_first_addresses(_f(blk["ra"]), _f(blk["rb"]), blk["L"])
        np.testing.assert_array_equal(got, np.array(blk["first"], np.int64))


def test_rmi_hand_leaf_predict():
    """Leaf of each key through the root, then the leaf's FP32 prediction: negative
    predictions clamp to 0, predictions past n-1 clamp to n-1, misrouted keys use the
    leaf the rounding picked (negative d)."""
    g = _rmi_hand()["leaf_predict"]
    r = g["root"]
    x = np.array([c["x"] for c in g["cases"]], np.uint32)
    leaf = rmi_ref.root_linear(_f(r["ra"]), _f(r["rb"]), x, r["L"])
    np.testing.assert_array_equal(leaf, np.array([c["leaf"] for c in g["cases"]]))
    a = np.array([_f(s) for s in g["a"]])
    b = np.array([_f(s) for s in g["b"]])
    x0 = np.array(g["x0"], np.int64)
    got = rmi_ref.leaf_predict(a, b, x0, leaf, x.astype(np.int64), g["n"])
    np.testing.assert_array_equal(got, np.array([c["pos"] for c in g["cases"]]))


def test_rmi_hand_eps_endpoints():
    """A one-leaf model that is exact in real arithmetic over-predicts by one just below
    each boundary because fl(x) rounds up to it: the bound is (1, 0) by hand."""
    g = _rmi_hand()["eps_endpoints_linear"]
    elo, ehi = rmi_ref.eps_endpoints_linear(np.array(g["starts"], np.uint32), _f(g["ra"]), _f(g["rb"]),
                                            np.array([_f(s) for s in g["a"]]), np.array([_f(s) for s in g["b"]]),
                                            np.array(g["x0"], np.int64), g["L"])
    np.testing.assert_array_equal(elo, g["eps_lo"])
    np.testing.assert_array_equal(ehi, g["eps_hi"])


def test_rmi_hand_leaf_predict_rounds_d():
    """The leaf-relative offset d is rounded to FP32 before the product: a hand case where
    that rounding decides the floor."""
    g = _rmi_hand()["leaf_predict_d_rounding"]
    x = np.array([c["x"] for c in g["cases"]], np.int64)
    leaf = np.zeros(x.size, np.int64)
    got = rmi_ref.leaf_predict(np.array([_f(s) for s in g["a"]]), np.array([_f(s) for s in g["b"]]),
                               np.array(g["x0"], np.int64), leaf, x, g["n"])
    np.testing.assert_array_equal(got, np.array([c["pos"] for c in g["cases"]]))


# --------------------------------------- learned index: minimax leaves, split leaves

def _lp_minimax(dlo, dhi, t):
    """The same minimax line as a linear programme (scipy's HiGHS): variables (a, c, E),
    minimise E subject to t - a dlo - c <= E, a dhi + c - t <= E, a >= 0."""
    linprog = pytest.importorskip("scipy.optimize").linprog
    dlo = np.asarray(dlo, np.float64)
    dhi = np.asarray(dhi, np.float64)
    t = np.asarray(t, np.float64)
    A = np.concatenate([np.stack([-dlo, -np.ones_like(dlo), -np.ones_like(dlo)], 1),
                        np.stack([dhi, np.ones_like(dhi), -np.ones_like(dhi)], 1)])
    ub = np.concatenate([-t, t])
    r = linprog([0, 0, 1], A_ub=A, b_ub=ub, bounds=[(0, None), (None, None), (None, None)], method="highs")
    assert r.status == 0
    return r.x[2]


def test_minimax_line_matches_linear_programme():
    """The ternary-search minimax fit reaches the optimum of the linear programme, on
    pieces that tile an interval (as a leaf's ranges do) and on scattered points."""
    rng = np.random.default_rng(7)
    for trial in range(60):
        k = int(rng.integers(1, 80))
        if trial % 2:
            cuts = np.sort(rng.choice(np.arange(1, 5000), size=k - 1, replace=False)) if k > 1 else np.zeros(0, int)
            lo = np.concatenate([[0], cuts])
            hi = np.concatenate([cuts, [5000]]) - 1
        else:
            lo = np.sort(rng.choice(np.arange(0, 10 ** 6), size=k, replace=False))
            hi = lo.copy()
        t = np.arange(k) + (rng.integers(0, 3, size=k).cumsum() if trial % 3 == 0 else 0)
        a, c, E = rmi_ref.minimax_line(lo, hi, t)
        assert a >= 0
        # the returned line achieves E, and E is the LP optimum
        got = max(np.max(t - (a * lo + c)), np.max(a * hi + c - t))
        assert got == pytest.approx(E, abs=1e-6)
        assert E == pytest.approx(_lp_minimax(lo, hi, t), abs=1e-6 * max(1.0, t.max()))


def test_minimax_line_closed_form():
    """k pieces of equal width w at positions 0..k-1: the best line is d / w with error
    (1 - 1/w) / 2 (the band is set by each piece's first and last address)."""
    for w in (1, 2, 7, 64, 1000):
        k = 37
        lo = np.arange(k) * w
        a, c, E = rmi_ref.minimax_line(lo, lo + w - 1, np.arange(k))
        assert E == pytest.approx((1 - 1 / w) / 2, abs=1e-9)
        assert a == pytest.approx(1 / w, rel=1e-9)


def test_route_models_by_hand():
    """Root leaves [0, 2^20), [2^20, 2^21), [2^21, 3*2^20), [3*2^20, 2^32) (ra = 4096); leaf 1
    split into 4 sub-leaves of 2^18 addresses (models 4..7), leaf 3 into 2 of 2^31 (models 8, 9)."""
    split = np.array([0, (3 << 8) | 18, 0, (1 << 8) | 31])
    first, lo, hi = rmi_ref.split_tables(4096.0, 0.0, 4, split)
    np.testing.assert_array_equal(first, [0, 1 << 20, 1 << 21, 3 << 20, 1 << 32])
    np.testing.assert_array_equal(lo[4:], [(1 << 20) + j * (1 << 18) for j in range(4)] + [3 << 20, (3 << 20) + (1 << 31)])
    np.testing.assert_array_equal(hi[4:], [(1 << 20) + (j + 1) * (1 << 18) for j in range(4)] + [(3 << 20) + (1 << 31), 1 << 32])
    x = np.array([0, (1 << 20) - 1, 1 << 20, (1 << 20) + (1 << 18) - 1, (1 << 20) + 3 * (1 << 18) + 5,
                  (1 << 21) - 1, 1 << 21, 3 << 20, (3 << 20) + (1 << 31) - 1, (3 << 20) + (1 << 31), 0xFFFFFFFF])
    want = [0, 0, 4, 4, 7, 7, 2, 8, 8, 9, 9]
    np.testing.assert_array_equal(rmi_ref.route_models(4096.0, 0.0, 4, split, first, x), want)


def test_eps_endpoints_models_by_brute_force():
    """Error bounds of a model with split leaves: without splits they equal the leaf-only
    analysis; with splits they equal the largest errors found by evaluating every address
    of [0, 2^20) and of the last 2^20 addresses, plus every model and range boundary +-1."""
    rng = np.random.default_rng(11)
    starts = np.unique(np.concatenate([[0], rng.integers(1, 1 << 20, 3000), [(1 << 32) - 5000]])).astype(np.int64)
    n = starts.size
    L = 8
    ra, rb = 8.0 * (1 << 12), 0.0          # leaves of 2^17 addresses up to 7 * 2^17, the rest in leaf 7
    split = np.zeros(L, np.int64)
    split[2] = (7 << 8) | 14               # 8 sub-leaves of 2^14
    split[7] = (3 << 8) | 30               # 4 sub-leaves over [7 * 2^17, 2^32)
    first, mlo, mhi = rmi_ref.split_tables(ra, rb, L, split)
    M = mlo.size
    a = np.zeros(M)
    b = np.zeros(M)
    x0 = np.minimum(mlo, (1 << 32) - 1)
    for m in range(M):
        if m < L and split[m]:
            continue
        am, bm, _ = rmi_ref.fit_interval_minimax(starts, int(mlo[m]), int(mhi[m]))
        a[m], b[m] = am, bm
    nosplit_lo, nosplit_hi = rmi_ref.eps_endpoints_models(starts, ra, rb, L, np.zeros(L, np.int64), a[:L], b[:L], x0[:L])
    ref_lo, ref_hi = rmi_ref.eps_endpoints_linear(starts, ra, rb, a[:L], b[:L], x0[:L], L)
    np.testing.assert_array_equal(nosplit_lo, ref_lo)
    np.testing.assert_array_equal(nosplit_hi, ref_hi)
    elo, ehi = rmi_ref.eps_endpoints_models(starts, ra, rb, L, split, a, b, x0)
    assert elo[2] == ehi[2] == elo[7] == ehi[7] == 0
    xs = np.concatenate([np.arange(0, 1 << 20), np.arange((1 << 32) - (1 << 20), 1 << 32), starts - 1, starts + 1,
                         mlo - 1, mlo, mhi - 1])
    xs = np.unique(xs[(xs >= 0) & (xs < (1 << 32))])
    model = rmi_ref.route_models(ra, rb, L, split, first, xs)
    t = np.searchsorted(starts, xs, side="right") - 1
    p = rmi_ref.leaf_predict(a, b, x0, model, xs, n)
    got_lo = np.zeros(M, np.int64)
    got_hi = np.zeros(M, np.int64)
    np.maximum.at(got_lo, model, np.maximum(p - t, 0))
    np.maximum.at(got_hi, model, np.maximum(t - p, 0))
    np.testing.assert_array_equal(got_lo, elo)
    np.testing.assert_array_equal(got_hi, ehi)
    # the minimax leaves keep every model's error near its optimum
    for m in range(M):
        if m < L and split[m]:
            continue
        E = rmi_ref.fit_interval_minimax(starts, int(mlo[m]), int(mhi[m]))[2]
        assert max(elo[m], ehi[m]) <= np.ceil(E + 0.5) + 1


def test_rate_stats_keys_equals_dense_rate_stats():
    """The per-key form of the rate statistics (for registries too large for a histogram
    per key) equals the histogram form on windows of the three registries, for every key
    with eligible flows and some without."""
    for reg, n, seed in ((fg.registry_c1(), 60_000, 5), (fg.registry_c2(), 60_000, 6)):
        rec = fg.make_records(reg, n, seed=seed)
        lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
        h, lo, hi, med = oracle.rate_stats(lpm, reg.local_prefix, reg.local_len, reg.n_sites, rec)
        keys = np.arange(2 * reg.n_sites)
        rmin, rmax, m, cnt = oracle.rate_stats_keys(lpm, reg.local_prefix, reg.local_len, reg.n_sites, rec, keys)
        np.testing.assert_array_equal(cnt, h.sum(axis=1))
        np.testing.assert_array_equal(m, med)
        np.testing.assert_array_equal(rmin, lo)
        np.testing.assert_array_equal(rmax, hi)
        assert (cnt > 0).sum() > 100 and (cnt == 0).sum() > 0
