"""Parity of the CUDA window path (through the C ABI) with the CPU oracle.

Integers (per-key flows, octets, packets, eligible flows/octets/durations, unmatched
classes, flags) must be bit-exact; rates within 1e-12 relative of the FP64 oracle.
"""
import ipaddress

import numpy as np
import pytest

import flowgen as fg
import oracle
from helpers import assert_rates_close, assert_window_matches, oracle_full
from test_oracle_pins import load_hand

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gnm():
    from paper_1108_1785_gb300 import build, gnm as g
    build.build()
    return g


@pytest.fixture(scope="module")
def c1():
    reg = fg.registry_c1()
    rec = fg.window_records_c1(reg)
    return reg, rec, oracle_full(reg, rec)


def _ctx(gnm, reg, **cfg):
    ctx = gnm.Context(**cfg)
    ctx.load(reg)
    return ctx


def test_hand_window(gnm):
    g, reg, loc, rec = load_hand()

    class R:
        pass
    r = R()
    r.prefix, r.plen, r.site = reg[:, 0], reg[:, 1], reg[:, 2]
    r.n_sites = g["n_sites"]
    r.local_prefix, r.local_len = loc[:, 0], loc[:, 1]
    for table in (gnm.TABLE_DIRECT, gnm.TABLE_HASH, gnm.TABLE_GLOBAL):
        ctx = _ctx(gnm, r, table_mode=table, threshold_bps=1e6)
        ctx.process(gnm.Records.to_device(rec), 7)
        st, un, rate, fl = ctx.dense(7)
        want = np.zeros_like(st)
        for row in g["expected_rows"]:
            want[row[0] * 2 + row[1]] = row[2:]
        np.testing.assert_array_equal(st, want)
        np.testing.assert_array_equal(un, np.array(g["expected_unmatched"], np.uint64))
        for key, v in g["expected_rates_bps"].items():
            s, d = map(int, key.split(","))
            assert rate[s * 2 + d] == pytest.approx(v, rel=1e-15)
        want_fl = np.zeros(st.shape[0], np.uint8)
        for s, d in g["thresholds"]["1e6"]:
            want_fl[s * 2 + d] = 1
        np.testing.assert_array_equal(fl, want_fl)
        sites, dirs = ctx.flag_suboptimal(7, 1e8)
        assert sorted(zip(sites.tolist(), dirs.tolist())) == sorted(map(tuple, g["thresholds"]["1e8"]))
        ctx.close()


# (BSEARCH, SMEM, bits): the ranges in shared memory behind a directory of `bits` bits (0: none;
# 16: too large to fit beside the ranges, so the whole range array is searched)
LOOKUPS = [("BSEARCH", "SMEM", 0), ("BSEARCH", "SMEM", 4), ("BSEARCH", "SMEM", 14), ("BSEARCH", "SMEM", 16),
           ("BSEARCH", "STAGED", 0), ("BSEARCH", "L2", 0), ("RADIX", "AUTO", 0), ("RADIX", "AUTO", 5)]
SPLITS = ["AUTO", "TWO_KERNELS"]


@pytest.mark.parametrize("table", ["DIRECT", "HASH", "GLOBAL"])
@pytest.mark.parametrize("agg", ["DIRECT", "WARP"])
@pytest.mark.parametrize("lookup", LOOKUPS, ids=lambda l: f"{l[0]}-{l[1]}-{l[2]}")
@pytest.mark.parametrize("unroll,block", [(1, 256), (2, 512), (1, 1024), (3, 768)])
@pytest.mark.parametrize("split", SPLITS)
def test_c1_window_all_variants(gnm, c1, table, agg, lookup, unroll, block, split):
    reg, rec, expect = c1
    mode, place, bits = lookup
    ctx = _ctx(gnm, reg, table_mode=getattr(gnm, "TABLE_" + table), aggregation=getattr(gnm, "AGG_" + agg),
               lookup_mode=getattr(gnm, "LOOKUP_" + mode), placement=getattr(gnm, "PLACE_" + place),
               radix_bits=bits, unroll=unroll, block_threads=block, hash_slots=512 if table == "HASH" else 0,
               split=getattr(gnm, "SPLIT_" + split))
    d = gnm.Records.to_device(rec)
    ctx.process(d, 1)
    assert_window_matches(ctx.dense(1), expect)
    # same window again into the same slot: identical
    ctx.process(d, 1)
    assert_window_matches(ctx.dense(1), expect)
    ctx.close()


def test_c1_host_records_and_site_stats(gnm, c1):
    reg, rec, expect = c1
    ctx = _ctx(gnm, reg)
    ctx.process(gnm.Records.host(rec), 3)  # host arrays: staged by the library
    assert_window_matches(ctx.dense(3), expect)
    rows, un = ctx.site_stats(3)
    ost = expect[0]
    active = np.nonzero(ost[:, 0])[0]
    assert [r.site * 2 + r.dir for r in rows] == active.tolist()
    for r in rows:
        k = r.site * 2 + r.dir
        assert [r.flows, r.octets, r.pkts, r.e_flows, r.e_octets, r.e_dur_ms] == ost[k].tolist()
        assert r.flag == expect[3][k]
    np.testing.assert_array_equal(un, expect[1])
    for thr in (1e5, 1e6, 3e6, 1e7, 1e8):
        sites, dirs = ctx.flag_suboptimal(3, thr)
        want = np.nonzero(oracle.flags(ost, expect[2], thr))[0]
        np.testing.assert_array_equal(sites.astype(np.int64) * 2 + dirs, want)
    ctx.close()


@pytest.mark.parametrize("split", ["FUSED", "TWO_KERNELS"])
def test_c1_ragged_and_unaligned(gnm, c1, split):
    """Windows of 0..9 records and arbitrary offsets (head/tail peeling), plus arrays
    whose 16-byte phases differ (element-wise path)."""
    reg, rec, _ = c1
    ctx = _ctx(gnm, reg, window_slots=128, split=getattr(gnm, "SPLIT_" + split))
    d = gnm.Records.to_device(rec)
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    wid = 100
    for start in (0, 1, 2, 3, 5, 4093):
        for n in (0, 1, 2, 3, 4, 5, 7, 9, 33, 1001):
            sub = {k: v[start:start + n] for k, v in d.fields.items()}
            ctx.process(gnm.Records(sub), wid)
            host = {k: v[start:start + n] for k, v in rec.items()}
            assert_window_matches(ctx.dense(wid), oracle_full(reg, host, lpm=lpm, n_threads=0))
            wid += 1
    # mixed phases: shift some fields by one element
    n = 5000
    fields = {}
    for j, k in enumerate(gnm.FIELDS):
        buf = torch.zeros(n + 4, dtype=torch.int32, device="cuda")
        off = j % 3
        buf[off:off + n] = d.fields[k][:n]
        fields[k] = buf[off:off + n]
    ctx.process(gnm.Records(fields), 999)
    host = {k: v[:n] for k, v in rec.items()}
    assert_window_matches(ctx.dense(999), oracle_full(reg, host, lpm=lpm))
    ctx.close()


@pytest.fixture(scope="module")
def c2hour():
    reg = fg.registry_c2()
    rec, off = fg.hour_records_c2(reg, seed=1)
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    expect = [oracle_full(reg, {k: v[off[w]:off[w + 1]] for k, v in rec.items()}, lpm=lpm) for w in range(60)]
    return reg, rec, off, expect


@pytest.mark.parametrize("cfg", [{}, {"split": "FUSED"}, {"lookup_mode": "BSEARCH"}, {"key_directory": 1},
                                 {"key_directory": 2}, {"key_directory": 3}, {"key_directory": 4}, {"key_directory": 3, "radix_bits": 8},
                                 {"key_directory": 1, "radix_bits": 15},
                                 {"key_directory": 1, "radix_bits": 4}, {"key_directory": 2, "radix_bits": 14},
                                 {"radix_bits": 10}, {"radix_bits": 4},
                                 {"lookup_mode": "BSEARCH", "placement": "L2", "split": "FUSED"},
                                 {"aggregation": "WARP"}, {"hash_slots": 1024}, {"table_mode": "GLOBAL"},
                                 {"radix_bits": 12, "split": "FUSED"}, {"table_mode": "HASH", "unroll": 2,
                                                                          "block_threads": 512},
                                 {"table_mode": "PARTITION"}, {"unroll": 3, "block_threads": 768},
                                 {"unroll": 3, "block_threads": 256}, {"table_mode": "PARTITION", "unroll": 3}])
def test_c2_hour_batched_bitexact(gnm, c2hour, cfg):
    """Sixty one-minute windows (10M records, nested registry) in one launch -- the
    benchmark's workload and, with cfg {}, its launch configuration; every window equals
    the oracle. Window 30 straddles the 32-bit millisecond wrap."""
    reg, rec, off, expect = c2hour
    kw = {}
    for k, v in cfg.items():
        kw[k] = getattr(gnm, {"placement": "PLACE_", "aggregation": "AGG_", "table_mode": "TABLE_",
                              "lookup_mode": "LOOKUP_", "split": "SPLIT_"}[k] + v) if isinstance(v, str) else v
    if "hash_slots" in kw:
        kw["table_mode"] = gnm.TABLE_HASH
    ctx = _ctx(gnm, reg, window_slots=64, **kw)
    if not cfg:  # the benchmark's default: radix-directed lookup, per-CTA shared-memory sums
        info = ctx.registry_info()
        assert info.lookup_mode == gnm.LOOKUP_RADIX and info.privatized
    d = gnm.Records.to_device(rec)
    ids = np.arange(60) + 5000
    plan = ctx.plan(d, off, ids)  # the benchmark's path: a CUDA graph of one launch
    plan.launch()
    # fused: one kernel; split: keys + sums; 10,004 keys: a grid-wide finalisation after them;
    # partitioned: keys (which also count the records of each bucket), scan, scatter, sums,
    # finalisation
    n_kernels = 5 if cfg.get("table_mode") == "PARTITION" else (1 if cfg.get("split") == "FUSED" else 2) + 1
    assert ctx.last_launch_count() == n_kernels
    for w in range(60):
        assert_window_matches(ctx.dense(int(ids[w])), expect[w])
    plan.close()
    ctx.close()


def test_windows_with_empty_and_many(gnm, c1):
    reg, rec, _ = c1
    ctx = _ctx(gnm, reg, window_slots=64)
    d = gnm.Records.to_device(rec)
    off = [0, 10, 10, 5000, 5001, 5001, 77777, 100000]
    ids = list(range(1, len(off)))
    ctx.process_windows(d, off, ids)
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    for w in range(len(ids)):
        host = {k: v[off[w]:off[w + 1]] for k, v in rec.items()}
        assert_window_matches(ctx.dense(ids[w]), oracle_full(reg, host, lpm=lpm, n_threads=0))
    ctx.close()


def test_open_add_close_equals_whole(gnm, c1):
    reg, rec, expect = c1
    ctx = _ctx(gnm, reg)
    d = gnm.Records.to_device(rec)
    ctx.open(11)
    cuts = [0, 1, 4097, 50000, 99999, 100000]
    for a, b in zip(cuts[:-1], cuts[1:]):
        ctx.add(gnm.Records({k: v[a:b] for k, v in d.fields.items()}), 11)
    with pytest.raises(gnm.GnmError):
        ctx.dense(11)  # still open
    ctx.close_window(11)
    assert_window_matches(ctx.dense(11), expect)
    ctx.close()


def test_slot_eviction_and_release(gnm, c1):
    reg, rec, expect = c1
    ctx = _ctx(gnm, reg, window_slots=2)
    d = gnm.Records.to_device(rec)
    ctx.process(d, 1)
    ctx.process(d, 2)
    ctx.process(d, 3)  # evicts window 1
    with pytest.raises(gnm.GnmError, match="STATE"):
        ctx.dense(1)
    assert_window_matches(ctx.dense(3), expect)
    ctx.release(2)
    with pytest.raises(gnm.GnmError, match="STATE"):
        ctx.dense(2)
    ctx.close()


@pytest.mark.parametrize("which,mode,place,bits", [("c1", "BSEARCH", "SMEM", 0), ("c1", "BSEARCH", "STAGED", 0),
                                                   ("c2", "BSEARCH", "STAGED", 0), ("c2", "BSEARCH", "L2", 0),
                                                   ("c1", "RADIX", "AUTO", 0), ("c2", "RADIX", "AUTO", 0),
                                                   ("c2", "RADIX", "AUTO", 4), ("c2", "RADIX", "AUTO", 15)])
# (gnm_lookup runs the batch lookup kernel; the window tests below cover the key kernel)
def test_lookup_matches_oracle(gnm, which, mode, place, bits):
    reg = fg.registry_c1() if which == "c1" else fg.registry_c2()
    ctx = _ctx(gnm, reg, lookup_mode=getattr(gnm, "LOOKUP_" + mode), placement=getattr(gnm, "PLACE_" + place),
               radix_bits=bits)
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    st, _ = lpm.flatten()
    s64 = st.astype(np.int64)
    x = np.concatenate([s64, s64 - 1, s64 + 1, [0, 0xFFFFFFFF],
                        np.random.default_rng(3).integers(0, 1 << 32, 200000)])
    x = x[(x >= 0) & (x < (1 << 32))].astype(np.uint32)
    dx = torch.from_numpy(x.view(np.int32)).cuda()
    site = torch.empty_like(dx)
    pos = torch.empty_like(dx)
    ctx.lookup(dx, site, pos)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(site.cpu().numpy().view(np.uint32), lpm.lookup(x))
    gst, gsi = ctx.ranges()
    np.testing.assert_array_equal(gst, st)  # the library's ranges equal the oracle's flattening
    np.testing.assert_array_equal(pos.cpu().numpy().view(np.uint32), np.searchsorted(st, x, side="right") - 1)
    ctx.close()


def _ip(s):
    return int(ipaddress.IPv4Address(s))


def test_radix_directory_must_fit(gnm):
    reg = fg.registry_c2()
    # one fused kernel would need a 256 KB 32-bit directory next to its sums
    ctx = _ctx(gnm, reg, lookup_mode=gnm.LOOKUP_RADIX, radix_bits=16, split=gnm.SPLIT_FUSED)
    d = gnm.Records.to_device(fg.make_records(reg, 1000, seed=3))
    with pytest.raises(gnm.GnmError, match="radix directory too large"):
        ctx.process(d, 1)
    ctx.close()


@pytest.mark.parametrize("which", ["c1", "c2"])
def test_hot_key_counts_do_not_wrap(gnm, which):
    """90% of 12M records share one (site, direction): every CTA's segment gives that key
    more than 2^16 records, so its 16-bit shared-memory counts must be handed over between
    pieces; the window still equals the oracle."""
    reg = fg.registry_c1() if which == "c1" else fg.registry_c2()
    rec = fg.make_records(reg, 12_000_000, seed=41)
    rng = np.random.default_rng(41)
    hot = rng.random(rec["srcaddr"].size) < 0.9
    inside = np.nonzero(reg.site == reg.site[0])[0][0]
    remote = np.uint32(int(reg.prefix[inside]) + 1)
    local = np.uint32(int(reg.local_prefix[0]) + 7)
    rec["srcaddr"] = np.where(hot, remote, rec["srcaddr"]).astype(np.uint32)
    rec["dstaddr"] = np.where(hot, local, rec["dstaddr"]).astype(np.uint32)
    ctx = _ctx(gnm, reg)
    ctx.process(gnm.Records.to_device(rec), 1)
    st, un, r, f = ctx.dense(1)
    assert st[:, 0].max() > 10_000_000  # the hot key
    assert_window_matches((st, un, r, f), oracle_full(reg, rec))
    ctx.close()


@pytest.mark.parametrize("cfg", [{}, {"table_mode": "PARTITION"}, {"table_mode": "HASH", "hash_slots": 1024},
                                 {"table_mode": "GLOBAL"}])
def test_one_slot_reused_after_global_sums(gnm, cfg):
    """One result slot for a sequence of windows: a hot key whose counts are handed to the
    global accumulators between pieces, 32-bit sums that wrap (octets near 2^32), a tiny
    window and a plain one. Finalisation reads only the accumulator groups that a launch
    wrote, and clears them, so every window equals the oracle."""
    reg = fg.registry_c2()
    kw = {k: getattr(gnm, "TABLE_" + v) if k == "table_mode" else v for k, v in cfg.items()}
    if kw.get("table_mode") == gnm.TABLE_PARTITION:
        reg = fg.registry_c3()
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    rng = np.random.default_rng(61)
    hot = fg.make_records(reg, 3_000_000, seed=62)
    pick = rng.random(hot["srcaddr"].size) < 0.8
    inside = np.nonzero(reg.site == reg.site[-1])[0][0]
    hot["srcaddr"] = np.where(pick, np.uint32(int(reg.prefix[inside]) + 1), hot["srcaddr"]).astype(np.uint32)
    hot["dstaddr"] = np.where(pick, np.uint32(int(reg.local_prefix[0]) + 9), hot["dstaddr"]).astype(np.uint32)
    big = fg.make_records(reg, 400_000, seed=63)
    big["dOctets"] = (np.uint32(0xFFFF0000) + (big["dOctets"] & np.uint32(0xFFFF))).astype(np.uint32)
    wins = [hot, big, fg.make_records(reg, 37, seed=64), fg.make_records(reg, 500_000, seed=65), hot]
    ctx = _ctx(gnm, reg, window_slots=1, **kw)
    for w, rec in enumerate(wins):
        ctx.process(gnm.Records.to_device(rec), 700 + w)
        assert_window_matches(ctx.dense(700 + w), oracle_full(reg, rec, lpm=lpm))
    ctx.close()


def test_rates_bit_exact_when_the_sums_pass_2_53(gnm):
    """2.5 M eligible flows of one (site, direction) with octets and durations near 2^32: the
    key's sums of eligible octets and durations pass 2^53, so converting them to FP64 rounds.
    The rates equal the FP64 oracle's bit for bit (the conversions and the x8000 are formed
    exactly on the integer units, the division is the FP64 one), on every key."""
    reg = fg.registry_c1()
    n = 2_500_000
    rec = fg.make_records(reg, n, seed=91)
    rng = np.random.default_rng(91)
    hot = rng.random(n) < 0.9
    inside = np.nonzero(reg.site == reg.site[3])[0][0]
    remote = np.uint32(int(reg.prefix[inside]) + 3)
    local = np.uint32(int(reg.local_prefix[0]) + 11)
    rec["srcaddr"] = np.where(hot, remote, rec["srcaddr"]).astype(np.uint32)
    rec["dstaddr"] = np.where(hot, local, rec["dstaddr"]).astype(np.uint32)
    big = (np.uint64(0xFFFFFFFF) - rng.integers(0, 1 << 24, size=n).astype(np.uint64)).astype(np.uint32)
    rec["dOctets"] = np.where(hot, big, rec["dOctets"]).astype(np.uint32)
    rec["dPkts"] = np.where(hot, rng.integers(10, 40, size=n), rec["dPkts"]).astype(np.uint32)
    dur = (np.uint64(0xFFFFFFFF) - rng.integers(0, 1 << 24, size=n).astype(np.uint64)).astype(np.uint32)
    rec["last"] = np.where(hot, rec["first"] + dur, rec["last"]).astype(np.uint32)  # mod 2^32
    ctx = _ctx(gnm, reg)
    ctx.process(gnm.Records.to_device(rec), 1)
    got = ctx.dense(1)
    want = oracle_full(reg, rec)
    key = int(reg.site[3]) * 2 + 0  # inbound: the remote end is the source
    assert want[0][key, 4] > 2 ** 53 and want[0][key, 5] > 2 ** 53
    assert_window_matches(got, want)
    gr, wr = np.asarray(got[2], np.float64), np.asarray(want[2], np.float64)
    np.testing.assert_array_equal(np.isnan(gr), np.isnan(wr))
    ok = ~np.isnan(wr)
    np.testing.assert_array_equal(gr[ok].view(np.uint64), wr[ok].view(np.uint64))
    ctx.close()


@pytest.mark.parametrize("which", ["c1", "c2"])
def test_host_records_in_place_and_staged(gnm, c1, which):
    """Page-locked host records read in place by the kernels, the same staged through a
    device copy, and pageable records (staged under AUTO, refused under IN_PLACE): every
    window equals the oracle."""
    reg = fg.registry_c1() if which == "c1" else fg.registry_c2()
    rec = fg.window_records_c1(reg, n=200_001) if which == "c1" else fg.make_records(reg, 200_001, seed=5)
    off = [0, 3, 100_000, 200_001]
    expect = [oracle_full(reg, {k: v[a:b] for k, v in rec.items()}) for a, b in zip(off[:-1], off[1:])]
    pinned = gnm.Records({k: torch.from_numpy(np.ascontiguousarray(rec[k]).view(np.int32)).pin_memory()
                          for k in gnm.FIELDS})
    pageable = gnm.Records.host(rec)
    for mode, recs, ok in (("IN_PLACE", pinned, True), ("STAGE", pinned, True), ("AUTO", pinned, True),
                           ("AUTO", pageable, True), ("IN_PLACE", pageable, False)):
        ctx = _ctx(gnm, reg, host_records=getattr(gnm, "HOST_" + mode))
        if not ok:
            with pytest.raises(gnm.GnmError, match="IN_PLACE"):
                ctx.process_windows(recs, off, [1, 2, 3])
        else:
            ctx.process_windows(recs, off, [1, 2, 3])
            for w, e in zip([1, 2, 3], expect):
                assert_window_matches(ctx.dense(w), e)
        ctx.close()


def test_host_records_pipelined(gnm):
    """PIPELINE: 12 windows (4.2 M records, with an empty one) copied in chunks of at least
    2^20 records to two alternating buffer sets while earlier chunks are processed; twice
    in a row (the buffers are reused) and from pageable arrays: every window equals the
    oracle."""
    reg = fg.registry_c2()
    rec = fg.make_records(reg, 4_200_000, seed=8)
    off = [0] + [350_000 * (w + 1) for w in range(12)]
    off[6] = off[5]  # window 5 empty
    expect = [oracle_full(reg, {k: v[a:b] for k, v in rec.items()}) for a, b in zip(off[:-1], off[1:])]
    pinned = gnm.Records({k: torch.from_numpy(np.ascontiguousarray(rec[k]).view(np.int32)).pin_memory()
                          for k in gnm.FIELDS})
    ctx = _ctx(gnm, reg, window_slots=32, host_records=gnm.HOST_PIPELINE)
    for rep, recs in enumerate((pinned, pinned, gnm.Records.host(rec))):
        ids = np.arange(12) + 100 * rep
        ctx.process_windows(recs, off, ids)
        for w in range(12):
            assert_window_matches(ctx.dense(int(ids[w])), expect[w])
    with pytest.raises(gnm.GnmError, match="duplicate"):
        ctx.process_windows(pinned, off, [1] * 12)
    ctx.close()


def test_partition_needs_split_launches(gnm):
    reg = fg.registry_c2()
    ctx = _ctx(gnm, reg, table_mode=gnm.TABLE_PARTITION, split=gnm.SPLIT_FUSED)
    d = gnm.Records.to_device(fg.make_records(reg, 1000, seed=3))
    with pytest.raises(gnm.GnmError, match="PARTITION needs split"):
        ctx.process(d, 1)
    ctx.close()


def test_block_samples_must_fit(gnm):
    reg = fg.registry_c2()
    # a 16-bit block directory (256 KB) and the block samples exceed one CTA's shared memory
    ctx = _ctx(gnm, reg, lookup_mode=gnm.LOOKUP_RADIX, radix_bits=16, key_directory=1)
    d = gnm.Records.to_device(fg.make_records(reg, 1000, seed=3))
    with pytest.raises(gnm.GnmError, match="block samples do not fit"):
        ctx.process(d, 1)
    ctx.close()


def test_sixteen_bit_block_directory_limits(gnm):
    """The 16-bit block directory holds block indices below 2^16: the 100,000-site registry
    (about 910,000 two-range blocks) refuses it when asked for and falls back to another
    directory by default; near the bucket edges (addresses t << 16 and t << 16 - 1 around
    registered prefixes) its lookups equal the oracle."""
    big = fg.registry_c3()
    d = gnm.Records.to_device(fg.make_records(big, 1000, seed=3))
    ctx = _ctx(gnm, big, lookup_mode=gnm.LOOKUP_RADIX, split=gnm.SPLIT_TWO_KERNELS, key_directory=4)
    with pytest.raises(gnm.GnmError, match="key_directory 4"):
        ctx.process(d, 1)
    ctx.close()
    reg = fg.registry_c2()
    rec = fg.make_records(reg, 200_000, seed=5)
    rng = np.random.default_rng(5)
    # remote ends on /16 bucket edges and on range starts and their predecessors
    starts, _ = gnm.registry_flatten(reg.prefix, reg.plen, reg.site, reg.n_sites)
    edges = np.concatenate([(np.arange(0, 1 << 16, dtype=np.uint64) << np.uint64(16)),
                            (np.arange(1, 1 << 16, dtype=np.uint64) << np.uint64(16)) - np.uint64(1),
                            starts.astype(np.uint64), starts[1:].astype(np.uint64) - np.uint64(1)])
    remote = edges[rng.integers(0, edges.size, size=rec["srcaddr"].size)].astype(np.uint32)
    inbound = rng.random(rec["srcaddr"].size) < 0.5
    local = np.uint32(int(reg.local_prefix[0]) + 5)
    rec["srcaddr"] = np.where(inbound, remote, local).astype(np.uint32)
    rec["dstaddr"] = np.where(inbound, local, remote).astype(np.uint32)
    ctx = _ctx(gnm, reg, lookup_mode=gnm.LOOKUP_RADIX, split=gnm.SPLIT_TWO_KERNELS, key_directory=4)
    ctx.process(gnm.Records.to_device(rec), 1)
    assert_window_matches(ctx.dense(1), oracle_full(reg, rec))
    ctx.close()


def test_registry_validation(gnm):
    ctx = gnm.Context()
    loc_p, loc_l = np.array([_ip("131.225.0.0")]), np.array([16])
    bad = [
        ([_ip("10.0.0.1")], [24], [0], 1, "host bits"),
        ([_ip("10.0.0.0")], [33], [0], 1, "length"),
        ([_ip("10.0.0.0")] * 2, [8, 8], [0, 0], 1, "duplicate"),
        ([_ip("10.0.0.0")], [8], [5], 1, "site id"),
        ([_ip("131.0.0.0")], [8], [0], 1, "overlaps"),
        ([_ip("131.225.7.0")], [24], [0], 1, "overlaps"),
    ]
    for p, l, s, ns, msg in bad:
        with pytest.raises(gnm.GnmError, match=msg):
            ctx.load_registry(np.array(p), np.array(l), np.array(s), ns, loc_p, loc_l)
    with pytest.raises(gnm.GnmError, match="STATE"):
        ctx.dense(0)
    ctx.close()


@pytest.fixture(scope="module")
def reg24():
    return fg.registry_c2_24()


@pytest.mark.parametrize("split", ["AUTO", "FUSED"])
def test_hash24_lookup_windows_match_oracle(gnm, reg24, split):
    """The paper's /24 subnet hash table as the lookup (registry of /8-/24 prefixes, 20%
    nested): windows equal the oracle and equal the binary-search lookup."""
    reg = reg24
    rec = fg.make_records(reg, 400_003, seed=13)
    off = [0, 150_000, 400_003]
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    ctx = _ctx(gnm, reg, lookup_mode=gnm.LOOKUP_HASH24, split=getattr(gnm, "SPLIT_" + split))
    assert ctx.registry_info().lookup_mode == gnm.LOOKUP_HASH24
    ctx.process_windows(gnm.Records.to_device(rec), off, [1, 2])
    for w, (a, b) in zip([1, 2], zip(off[:-1], off[1:])):
        assert_window_matches(ctx.dense(w), oracle_full(reg, {k: v[a:b] for k, v in rec.items()}, lpm=lpm))
    ctx.close()


def test_hash24_batch_lookup_and_limits(gnm, reg24):
    reg = reg24
    ctx = _ctx(gnm, reg, lookup_mode=gnm.LOOKUP_HASH24)
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    st, _ = lpm.flatten()
    s64 = st.astype(np.int64)
    x = np.concatenate([s64, s64 - 1, s64 + 1, s64 + 255, [0, 0xFFFFFFFF],
                        np.random.default_rng(8).integers(0, 1 << 32, 300_000)])
    x = x[(x >= 0) & (x < (1 << 32))].astype(np.uint32)
    dx = torch.from_numpy(x.view(np.int32)).cuda()
    site = torch.empty_like(dx)
    ctx.lookup(dx, site)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(site.cpu().numpy().view(np.uint32), lpm.lookup(x))
    with pytest.raises(gnm.GnmError, match="positions"):
        ctx.lookup(dx, site, torch.empty_like(dx))
    ctx.close()
    longer = _ctx(gnm, fg.registry_c2(), lookup_mode=gnm.LOOKUP_HASH24)  # has /25-/30 prefixes
    with pytest.raises(gnm.GnmError, match="longer than /24"):
        longer.process(gnm.Records.to_device(fg.make_records(fg.registry_c2(), 1000, seed=2)), 1)
    longer.close()


@pytest.mark.parametrize("n_sites", [4999, 2001])
def test_odd_site_count_windows_equal_oracle(gnm, n_sites):
    """Registries with an odd number of sites (2 * n_sites + 4 keys, not a multiple of four):
    the aggregation stores its partial blocks word by word instead of in 16-byte column
    words. Three windows of 700,000 records each (many CTAs per window, several count
    hand-overs per CTA), split launches and one fused launch, every window equal to the
    oracle."""
    reg = fg.make_registry(n_sites, 8 * n_sites, fg.C2_LEN, 0.2, seed=n_sites)
    recs = [fg.make_records(reg, 700_000, seed=n_sites + k, p_reg=0.85, zipf_s=1.0) for k in range(3)]
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    for cfg in ({}, {"split": gnm.SPLIT_FUSED, "lookup_mode": gnm.LOOKUP_BSEARCH, "placement": gnm.PLACE_L2}):
        ctx = _ctx(gnm, reg, window_slots=8, **cfg)
        for w, rec in enumerate(recs):
            ctx.process(gnm.Records.to_device(rec), 40 + w)
            assert_window_matches(ctx.dense(40 + w), oracle_full(reg, rec, lpm=lpm))
        ctx.close()
