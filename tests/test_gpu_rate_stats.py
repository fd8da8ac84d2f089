"""Per-flow rate statistics (Sec. III.B.2.1: minimum, maximum, and the median from a
histogram of 10 kb/s buckets) against the oracle: histograms and median buckets bit-exact,
minimum and maximum rates bit-exact (the same FP64 operations in the same order)."""
import numpy as np
import pytest

import flowgen as fg
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gnm():
    from paper_1108_1785_gb300 import build, gnm as g
    build.build()
    return g


def _expect(reg, rec, lpm=None):
    lpm = lpm or oracle.LPM(reg.prefix, reg.plen, reg.site)
    return oracle.rate_stats(lpm, reg.local_prefix, reg.local_len, reg.n_sites, rec)


def _check(got, want):
    rmin, rmax, med, hist = got
    h, lo, hi, m = want
    np.testing.assert_array_equal(hist, h)
    np.testing.assert_array_equal(med, m)
    np.testing.assert_array_equal(rmin, lo)  # NaN where there is no eligible flow, on both sides
    np.testing.assert_array_equal(rmax, hi)


@pytest.mark.parametrize("which,cfg", [("c1", {}),                                   # fused, direct table
                                       ("c2", {}),                                   # split, direct table
                                       ("c2", {"table_mode": "PARTITION"}),          # regrouped records
                                       ("c2", {"table_mode": "HASH", "split": "FUSED"})])
def test_rate_stats_match_oracle(gnm, which, cfg):
    reg = fg.registry_c1() if which == "c1" else fg.registry_c2()
    rec = fg.make_records(reg, 600_001, seed=17)
    off = [0, 250_000, 600_001]
    kw = {k: getattr(gnm, {"table_mode": "TABLE_", "split": "SPLIT_"}[k] + v) for k, v in cfg.items()}
    ctx = gnm.Context(window_slots=4, rate_stats=1, **kw)
    ctx.load(reg)
    plan = ctx.plan(gnm.Records.to_device(rec), off, [3, 4])
    for _ in range(2):  # replays clear the statistics first
        plan.launch()
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    for w, (a, b) in zip([3, 4], zip(off[:-1], off[1:])):
        _check(ctx.rate_stats(w, hist=True), _expect(reg, {k: v[a:b] for k, v in rec.items()}, lpm))
    plan.close()
    ctx.close()


def test_rate_stats_open_add_close_and_refusal(gnm):
    reg = fg.registry_c1()
    rec = fg.window_records_c1(reg, n=90_000)
    ctx = gnm.Context(window_slots=4, rate_stats=1)
    ctx.load(reg)
    d = gnm.Records.to_device(rec)
    ctx.open(9)
    for a, b in ((0, 1), (1, 40_000), (40_000, 90_000)):
        ctx.add(gnm.Records({k: v[a:b] for k, v in d.fields.items()}), 9)
    ctx.close_window(9)
    _check(ctx.rate_stats(9, hist=True), _expect(reg, rec))
    ctx.process(d, 9)  # the same id again: the statistics start over
    _check(ctx.rate_stats(9, hist=True), _expect(reg, rec))
    ctx.close()
    off = gnm.Context(window_slots=2)
    off.load(reg)
    off.process(d, 1)
    with pytest.raises(gnm.GnmError, match="STATE"):
        off.rate_stats(1)
    off.close()


@pytest.mark.parametrize("consecutive", [1, 2, 3])
def test_warnings_follow_oracle_over_windows(gnm, consecutive):
    """Five windows in time order: after each, the keys whose median bucket stayed below 100
    (1 Mb/s) for `consecutive` windows in a row equal the oracle's warnings; a reset starts
    every run over."""
    reg = fg.registry_c1()
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    wins = [fg.make_records(reg, 60_000, seed=100 + w, zipf_s=1.1) for w in range(5)]
    meds = [_expect(reg, r, lpm)[3] for r in wins]
    want = oracle.warnings(meds, below_bucket=100, consecutive=consecutive)
    ctx = gnm.Context(window_slots=8, rate_stats=1)
    ctx.load(reg)
    for w, r in enumerate(wins):
        ctx.process(gnm.Records.to_device(r), 50 + w)
        got = ctx.warnings_update(50 + w, below_bucket=100, consecutive=consecutive)
        np.testing.assert_array_equal(got, np.nonzero(want[w])[0])
    assert any(x.any() for x in want)  # the workload does raise warnings
    ctx.warnings_reset()
    got = ctx.warnings_update(54, below_bucket=100, consecutive=consecutive)
    np.testing.assert_array_equal(got, np.nonzero(oracle.warnings(meds[4:], consecutive=consecutive)[0])[0])
    ctx.close()


def test_warnings_resume_from_exported_runs(gnm):
    """Monitoring stopped after window 2 and resumed in a new context from the exported runs
    gives, for windows 3 and 4, the warnings of the uninterrupted sequence."""
    reg = fg.registry_c1()
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    wins = [fg.make_records(reg, 60_000, seed=200 + w, zipf_s=1.1) for w in range(5)]
    want = oracle.warnings([_expect(reg, r, lpm)[3] for r in wins], below_bucket=100, consecutive=2)
    first = gnm.Context(window_slots=4, rate_stats=1)
    first.load(reg)
    for w in range(3):
        first.process(gnm.Records.to_device(wins[w]), w)
        first.warnings_update(w)
    runs = first.warnings_export()
    first.close()
    second = gnm.Context(window_slots=4, rate_stats=1)
    second.load(reg)
    second.warnings_import(runs)
    for w in (3, 4):
        second.process(gnm.Records.to_device(wins[w]), w)
        np.testing.assert_array_equal(second.warnings_update(w), np.nonzero(want[w])[0])
    second.close()


# ------------------------------------------------------------ sparse (rate_stats = 2)

def _cells_of(hist):
    k, b = np.nonzero(hist)
    return k.astype(np.uint32), b.astype(np.uint32), hist[k, b].astype(np.uint32)


@pytest.mark.parametrize("which,cfg", [("c1", {}),                                   # fused, direct table
                                       ("c2", {}),                                   # split, direct table
                                       ("c2", {"table_mode": "PARTITION"}),          # regrouped records
                                       ("c2", {"table_mode": "HASH", "split": "FUSED"})])
def test_sparse_rate_stats_match_oracle(gnm, which, cfg):
    """The sparse log (one word per eligible flow, sorted on the GPU when read) gives the
    oracle's medians, least and greatest rates, and its cells are the non-empty cells of the
    oracle's histograms, in every launch kind and on plan replays."""
    reg = fg.registry_c1() if which == "c1" else fg.registry_c2()
    rec = fg.make_records(reg, 600_001, seed=17)
    off = [0, 250_000, 600_001]
    kw = {k: getattr(gnm, {"table_mode": "TABLE_", "split": "SPLIT_"}[k] + v) for k, v in cfg.items()}
    ctx = gnm.Context(window_slots=4, rate_stats=2, **kw)
    ctx.load(reg)
    plan = ctx.plan(gnm.Records.to_device(rec), off, [3, 4])
    for _ in range(2):  # replays clear the log first
        plan.launch()
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    for w, (a, b) in zip([3, 4], zip(off[:-1], off[1:])):
        h, lo, hi, m = _expect(reg, {k: v[a:b] for k, v in rec.items()}, lpm)
        rmin, rmax, med, none = ctx.rate_stats(w)
        assert none is None
        np.testing.assert_array_equal(med, m)
        np.testing.assert_array_equal(rmin, lo)
        np.testing.assert_array_equal(rmax, hi)
        for got, want in zip(ctx.rate_cells(w), _cells_of(h)):
            np.testing.assert_array_equal(got, want)
    with pytest.raises(gnm.GnmError, match="INVAL"):
        ctx.rate_stats(3, hist=True)
    plan.close()
    ctx.close()


def test_sparse_log_grows_across_adds(gnm):
    """A window filled by several adds outgrows its first log (65,536 words): the log grows,
    keeps the words logged so far, and the statistics equal the dense histograms'."""
    reg = fg.registry_c1()
    rec = fg.window_records_c1(reg, n=300_000)
    d = gnm.Records.to_device(rec)
    out = {}
    for mode in (1, 2):
        ctx = gnm.Context(window_slots=4, rate_stats=mode)
        ctx.load(reg)
        ctx.open(9)
        for a, b in ((0, 1), (1, 50_000), (50_000, 120_001), (120_001, 300_000)):
            ctx.add(gnm.Records({k: v[a:b] for k, v in d.fields.items()}), 9)
        ctx.close_window(9)
        out[mode] = (ctx.rate_stats(9)[:3], ctx.rate_cells(9))
        ctx.close()
    for a, b in zip(out[1][0], out[2][0]):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(out[1][1], out[2][1]):
        np.testing.assert_array_equal(a, b)
    _, lo, hi, m = _expect(reg, rec)
    np.testing.assert_array_equal(out[2][0][2], m)


def test_sparse_warnings_equal_dense(gnm):
    """Median warnings over five windows are the same with the sparse log."""
    reg = fg.registry_c1()
    wins = [fg.make_records(reg, 60_000, seed=300 + w, zipf_s=1.1) for w in range(5)]
    got = {}
    for mode in (1, 2):
        ctx = gnm.Context(window_slots=8, rate_stats=mode)
        ctx.load(reg)
        got[mode] = []
        for w, r in enumerate(wins):
            ctx.process(gnm.Records.to_device(r), w)
            got[mode].append(ctx.warnings_update(w, below_bucket=100, consecutive=2))
        ctx.close()
    for a, b in zip(got[1], got[2]):
        np.testing.assert_array_equal(a, b)
    assert any(len(a) for a in got[1])


def test_sparse_rate_stats_site_limit(gnm):
    """Keys of the sparse log have 18 bits: registries of more than 131,072 sites are refused
    at load time."""
    n = 131_073
    reg = fg.Registry(prefix=(np.arange(n, dtype=np.uint32) << 8) + np.uint32(1 << 24),
                      plen=np.full(n, 24, np.uint8), site=np.arange(n, dtype=np.uint32), n_sites=n,
                      local_prefix=np.array([0xC0A80000], np.uint32), local_len=np.array([16], np.uint8),
                      holes=np.zeros((0, 2), np.int64), nested=np.zeros(n, bool))
    ctx = gnm.Context(window_slots=2, rate_stats=2)
    with pytest.raises(gnm.GnmError, match="131,072"):
        ctx.load(reg)
    ctx.close()
