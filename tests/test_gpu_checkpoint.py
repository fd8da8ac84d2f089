"""Checkpoint of an open window (gnm_window_export / gnm_window_import): a window whose
first records were added in one context, exported, imported into another context over the
same registry and finished there equals the whole window processed at once -- integers
bit-exact, rates within 1e-12 -- and the CPU oracle."""
import numpy as np
import pytest

import flowgen as fg
from helpers import assert_rates_close, assert_window_matches, oracle_full

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gnm():
    from paper_1108_1785_gb300 import build, gnm as g
    build.build()
    return g


def _ctx(gnm, reg, **cfg):
    ctx = gnm.Context(**cfg)
    ctx.load(reg)
    return ctx


def _slice(d, a, b, gnm):
    return gnm.Records({k: v[a:b] for k, v in d.fields.items()})


@pytest.mark.parametrize("which,cfg", [("c1", {}), ("c2", {}), ("c2", {"split": "FUSED"}), ("c3", {})])
def test_resume_in_another_context_equals_whole(gnm, which, cfg):
    reg = {"c1": fg.registry_c1, "c2": fg.registry_c2, "c3": fg.registry_c3}[which]()
    rec = fg.make_records(reg, 700_003, seed=81)
    d = gnm.Records.to_device(rec)
    kw = {k: getattr(gnm, "SPLIT_" + v) for k, v in cfg.items()}
    first = _ctx(gnm, reg, window_slots=4, **kw)
    first.open(5)
    for a, b in ((0, 1), (1, 250_000), (250_000, 400_000)):
        first.add(_slice(d, a, b, gnm), 5)
    rows = first.window_export(5)
    assert rows.shape == (2 * reg.n_sites + 4, 6)
    assert int(rows[:, 0].sum()) == 400_000  # every record lands in one key
    first.close_window(5)  # the exporting context can still finish its own copy
    second = _ctx(gnm, reg, window_slots=4, **kw)
    second.window_import(9, rows)
    second.add(_slice(d, 400_000, 700_003, gnm), 9)
    second.close_window(9)
    whole = _ctx(gnm, reg, window_slots=4, **kw)
    whole.process(d, 1)
    got, want = second.dense(9), whole.dense(1)
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])
    assert_rates_close(got[2], want[2])
    np.testing.assert_array_equal(got[3], want[3])
    if which == "c1":
        assert_window_matches(got, oracle_full(reg, rec))
    # the first context's window holds only the first 400,000 records
    part = {k: v[:400_000] for k, v in rec.items()}
    whole.process(gnm.Records.to_device(part), 2)
    np.testing.assert_array_equal(first.dense(5)[0], whole.dense(2)[0])
    for c in (first, second, whole):
        c.close()


def test_export_import_round_trip_and_errors(gnm):
    reg = fg.registry_c1()
    rec = fg.make_records(reg, 100_000, seed=82)
    d = gnm.Records.to_device(rec)
    ctx = _ctx(gnm, reg, window_slots=4)
    ctx.open(1)
    ctx.add(d, 1)
    rows = ctx.window_export(1)
    ctx.window_import(2, rows)  # a copy in the same context
    np.testing.assert_array_equal(ctx.window_export(2), rows)
    ctx.close_window(1)
    ctx.close_window(2)
    for x, y in zip(ctx.dense(1), ctx.dense(2)):
        np.testing.assert_array_equal(x, y)
    with pytest.raises(gnm.GnmError, match="STATE"):
        ctx.window_export(1)  # closed
    with pytest.raises(gnm.GnmError, match="STATE"):
        ctx.window_export(77)  # unknown
    bad = rows.copy()
    bad[0, 3] = bad[0, 0] + 1  # e_flows above flows
    with pytest.raises(gnm.GnmError, match="INVAL"):
        ctx.window_import(3, bad)
    bad = rows.copy()
    bad[1, 4] = bad[1, 1] + 1  # e_octets above octets
    with pytest.raises(gnm.GnmError, match="INVAL"):
        ctx.window_import(3, bad)
    with pytest.raises(gnm.GnmError, match="INVAL"):
        ctx.window_import(3, rows[:-1])
    ctx.close()
    stats = _ctx(gnm, reg, window_slots=4, rate_stats=1)
    stats.open(1)
    stats.add(d, 1)
    with pytest.raises(gnm.GnmError, match="STATE"):
        stats.window_export(1)
    with pytest.raises(gnm.GnmError, match="STATE"):
        stats.window_import(2, rows)
    stats.close()
