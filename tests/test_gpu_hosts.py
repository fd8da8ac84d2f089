"""Per-host sums (Sec. III.B.2.1: statistics for each host in a registered site) against the
oracle: one row per (remote address, direction) of a registered site, sums bit-exact, the
site from the longest-prefix match, rates within 1e-12 (the same FP64 formula)."""
import numpy as np
import pytest

import flowgen as fg
import oracle
from helpers import assert_rates_close

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gnm():
    from paper_1108_1785_gb300 import build, gnm as g
    build.build()
    return g


@pytest.mark.parametrize("which,cfg", [("c1", {}), ("c2", {}), ("c2", {"table_mode": "PARTITION"})])
def test_host_rows_match_oracle(gnm, which, cfg):
    reg = fg.registry_c1() if which == "c1" else fg.registry_c2()
    rec = fg.make_records(reg, 500_001, seed=23)
    off = [0, 200_000, 500_001]
    kw = {k: getattr(gnm, "TABLE_" + v) for k, v in cfg.items()}
    ctx = gnm.Context(window_slots=4, host_capacity=300_000, **kw)
    ctx.load(reg)
    plan = ctx.plan(gnm.Records.to_device(rec), off, [5, 6])
    for _ in range(2):  # replays clear the tables first
        plan.launch()
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    for w, (a, b) in zip([5, 6], zip(off[:-1], off[1:])):
        addr, site, d, sums, rate = ctx.hosts(w)
        ea, es, ed, esums = oracle.host_stats(lpm, reg.local_prefix, reg.local_len, reg.n_sites,
                                              {k: v[a:b] for k, v in rec.items()})
        np.testing.assert_array_equal(addr, ea)
        np.testing.assert_array_equal(site, es)
        np.testing.assert_array_equal(d, ed)
        np.testing.assert_array_equal(sums, esums)
        assert_rates_close(rate, oracle.rates(esums))
    plan.close()
    ctx.close()


def test_host_table_limits(gnm):
    reg = fg.registry_c1()
    rec = fg.window_records_c1(reg, n=50_000)
    d = gnm.Records.to_device(rec)
    small = gnm.Context(window_slots=2, host_capacity=100)  # far fewer entries than hosts
    small.load(reg)
    small.process(d, 1)
    with pytest.raises(gnm.GnmError, match="CAPACITY"):
        small.hosts(1)
    small.close()
    fused = gnm.Context(window_slots=2, host_capacity=1000, split=gnm.SPLIT_FUSED)
    fused.load(reg)
    with pytest.raises(gnm.GnmError, match="split launches"):
        fused.process(d, 1)
    fused.close()
    off = gnm.Context(window_slots=2)
    off.load(reg)
    off.process(d, 1)
    with pytest.raises(gnm.GnmError, match="STATE"):
        off.hosts(1)
    off.close()
