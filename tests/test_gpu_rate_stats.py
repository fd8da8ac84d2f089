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
