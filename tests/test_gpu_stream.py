"""Streaming server (gnm_stream_*): every window's result is the same when its batches are
served in a mix with other windows' batches -- interleaved, queued under a memory budget,
spread over several CUDA streams -- as when the window is processed alone; sampled windows
also match the CPU oracle. Integers bit-exact, rates within 1e-12 relative."""
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


@pytest.fixture(scope="module")
def regs():
    # c3: 100,000 sites (200,004 keys): each batch regroups its records by key group
    return {"c1": fg.registry_c1(), "c2": fg.registry_c2(), "c3": fg.registry_c3()}


def _ctx(gnm, reg, **cfg):
    ctx = gnm.Context(**cfg)
    ctx.load(reg)
    return ctx


def _plan_mix(rng, n_windows, pool_n, max_batch, empty_close_every=4):
    """Per window a list of pool slices (a, b); a submission order that interleaves the
    windows while keeping each window's batches in order; the last batch closes."""
    sizes_pick = [0, 1, 3, 17, 4096]
    wins = {}
    for w in range(n_windows):
        k = int(rng.integers(2, 7))
        sl = []
        for _ in range(k):
            n = int(rng.choice(sizes_pick)) if rng.random() < 0.3 else int(rng.integers(1, max_batch + 1))
            a = int(rng.integers(0, pool_n - n + 1))
            sl.append((a, a + n))
        wins[100 + w] = sl
    order = []
    left = {w: list(range(len(s))) for w, s in wins.items()}
    while left:
        w = int(rng.choice(sorted(left)))
        order.append((w, left[w].pop(0)))
        if not left[w]:
            del left[w]
    empty_close = {w for i, w in enumerate(sorted(wins)) if i % empty_close_every == 0}
    return wins, order, empty_close


def _pinned(pool):
    """The pool in page-locked host memory (numpy views of pinned tensors, kept alive by the
    returned tensors)."""
    t = {k: torch.from_numpy(np.ascontiguousarray(pool[k]).view(np.int32)).pin_memory() for k in fg.FIELDS}
    return t, {k: v.numpy().view(np.uint32) for k, v in t.items()}


def _concat(pool, slices):
    return {k: np.concatenate([v[a:b] for a, b in slices]) for k, v in pool.items()}


def _serve(gnm, stream, pool_recs, wins, order, empty_close, read):
    """Submits in `order`; `read(wid)` is called for each reported window before the next
    server call (its results are guaranteed on the device until then)."""
    done = {}
    for w, j in order:
        a, b = wins[w][j]
        last = j == len(wins[w]) - 1
        stream.submit(pool_recs(a, b), w, close=last and w not in empty_close)
        if last and w in empty_close:
            stream.close_window(w)
        for wid, n, lat, status in stream.poll():
            done[wid] = (n, lat, status, read(wid))
    while len(done) < len(wins):
        for wid, n, lat, status in stream.poll(wait_all=True):
            done[wid] = (n, lat, status, read(wid))
    return done


@pytest.mark.parametrize("which,host,budget_batches,n_streams,slots", [
    ("c1", True, 2, 3, 64),     # fused launches, host batches copied into the arena
    ("c2", True, 3, 4, 64),     # split (key + aggregation) launches
    ("c1", False, 2, 2, 64),    # device batches: only the budget is charged
    ("c2", True, 2, 4, 3),      # three result slots for twelve interleaved windows
    ("c3", True, 3, 4, 8),      # a key space larger than one shared-memory table
    ("c2", "pinned", 3, 4, 64),  # page-locked host batches: read in place by the kernels
    ("c3", "pinned", 3, 4, 8),
])
def test_mix_equals_alone(gnm, regs, which, host, budget_batches, n_streams, slots):
    reg = regs[which]
    rng = np.random.default_rng(11)
    pool = fg.make_records(reg, 300_000, seed=21)
    max_batch = 30_000
    wins, order, empty_close = _plan_mix(rng, 12, 300_000, max_batch)
    if host == "pinned":
        hold, ppool = _pinned(pool)

        def recs(a, b):
            return gnm.Records({k: v[a:b] for k, v in ppool.items()})
    elif host:
        def recs(a, b):
            return gnm.Records.host({k: v[a:b] for k, v in pool.items()})
    else:
        dpool = gnm.Records.to_device(pool)

        def recs(a, b):
            return gnm.Records({k: v[a:b] for k, v in dpool.fields.items()})
    ctx = _ctx(gnm, reg, window_slots=slots)
    budget = budget_batches * max_batch * 24
    stream = gnm.Stream(ctx, budget_bytes=budget, n_cuda_streams=n_streams)
    done = _serve(gnm, stream, recs, wins, order, empty_close, ctx.dense)
    st = stream.stats()
    stream.close()
    assert sorted(done) == sorted(wins)
    assert st["peak_inflight_bytes"] <= budget
    assert st["inflight_bytes"] == 0
    assert st["windows_done"] == len(wins) and st["batches"] == len(order) + len(empty_close)
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    alone = _ctx(gnm, reg)
    for w, sl in wins.items():
        n, lat, status, dense = done[w]
        assert status == 0 and lat > 0
        rec = _concat(pool, sl)
        assert n == rec["srcaddr"].size
        alone.process(gnm.Records.to_device(rec), w)
        st_a, un_a, r_a, f_a = alone.dense(w)
        np.testing.assert_array_equal(dense[0], st_a)
        np.testing.assert_array_equal(dense[1], un_a)
        assert_rates_close(dense[2], r_a)
        np.testing.assert_array_equal(dense[3], f_a)
    for w in sorted(wins)[::5]:  # sampled windows against the oracle
        assert_window_matches(done[w][3], oracle_full(reg, _concat(pool, wins[w])))
    alone.close()
    ctx.close()


def test_empty_window_and_reuse_of_an_id(gnm, regs):
    reg = regs["c1"]
    ctx = _ctx(gnm, reg)
    stream = gnm.Stream(ctx, budget_bytes=1 << 20)
    stream.close_window(5)  # never received a record
    (wid, n, lat, status), = stream.poll(wait_all=True)
    assert (wid, n, status) == (5, 0, 0)
    st, un, r, f = ctx.dense(5)
    assert not st.any() and not un.any() and np.isnan(r).all() and not f.any()
    pool = fg.window_records_c1(reg, n=5000)
    stream.submit(gnm.Records.host(pool), 5, close=True)  # the id is free again once reported
    (wid, n, lat, status), = stream.poll(wait_all=True)
    assert (wid, n, status) == (5, 5000, 0)
    assert_window_matches(ctx.dense(5), oracle_full(reg, pool))
    stream.close()
    ctx.close()


def test_admission_errors_and_slot_wait(gnm, regs):
    reg = regs["c1"]
    ctx = _ctx(gnm, reg, window_slots=1)
    pool = fg.window_records_c1(reg, n=4000)
    part = lambda a, b: gnm.Records.host({k: v[a:b] for k, v in pool.items()})  # noqa: E731
    stream = gnm.Stream(ctx, budget_bytes=2000 * 24, max_queued=2)
    with pytest.raises(gnm.GnmError, match="INVAL"):
        stream.submit(part(0, 2001), 1)  # larger than the whole budget
    stream.submit(part(0, 1000), 1)      # window 1 takes the only slot
    stream.submit(part(1000, 2000), 2)   # waits for a slot
    stream.submit(part(2000, 3000), 3)   # waits too: the queue is full now
    with pytest.raises(gnm.GnmError, match="CAPACITY"):
        stream.submit(part(3000, 4000), 4)
    with pytest.raises(gnm.GnmError, match="STATE"):
        stream.poll(wait_all=True)       # only closing window 1 frees the slot
    assert stream.stats()["batches_queued"] == 2
    stream.close_window(1)
    with pytest.raises(gnm.GnmError, match="STATE"):
        stream.submit(part(0, 10), 1)    # a closed window takes no more batches
    got = stream.poll(wait_all=True)     # window 1 done; 2 waits for its slot until the next call
    assert [g[0] for g in got] == [1]
    assert_window_matches(ctx.dense(1), oracle_full(reg, {k: v[0:1000] for k, v in pool.items()}))
    stream.close_window(2)
    stream.close_window(3)
    seen = {}
    while len(seen) < 2:
        for wid, n, lat, status in stream.poll(wait_all=True):
            seen[wid] = ctx.dense(wid)
    for wid, (a, b) in ((2, (1000, 2000)), (3, (2000, 3000))):
        assert_window_matches(seen[wid], oracle_full(reg, {k: v[a:b] for k, v in pool.items()}))
    st = stream.stats()
    assert st["peak_inflight_bytes"] <= 2000 * 24 and st["windows_done"] == 3
    stream.close()
    ctx.close()


def test_window_of_a_plan_fails_alone(gnm, regs):
    """A window whose slot cannot be taken (its id belongs to a plan) is reported with the
    error; the other windows of the mix are unaffected."""
    reg = regs["c1"]
    ctx = _ctx(gnm, reg)
    pool = fg.window_records_c1(reg, n=20000)
    d = gnm.Records.to_device(pool)
    plan = ctx.plan(d, [0, 10000], [77])
    stream = gnm.Stream(ctx, budget_bytes=1 << 22)
    stream.submit(gnm.Records.host({k: v[:5000] for k, v in pool.items()}), 77, close=True)
    stream.submit(gnm.Records.host({k: v[5000:] for k, v in pool.items()}), 78, close=True)
    got = {}
    while len(got) < 2:
        for wid, n, lat, status in stream.poll(wait_all=True):
            got[wid] = status
            if status == 0:
                assert_window_matches(ctx.dense(wid), oracle_full(reg, {k: v[5000:] for k, v in pool.items()}))
    assert got[77] == 4 and got[78] == 0  # GNM_E_STATE for the plan's window
    stream.close()
    plan.close()
    ctx.close()


def test_served_windows_keep_rate_and_host_statistics(gnm, regs):
    """A context that also keeps per-flow rate statistics and per-host sums: every served
    window (interleaved batches) has the same statistics as the window processed alone."""
    reg = regs["c2"]
    rng = np.random.default_rng(19)
    pool = fg.make_records(reg, 200_000, seed=29)
    wins, order, empty_close = _plan_mix(rng, 6, 200_000, 20_000)
    cfg = dict(window_slots=16, rate_stats=1, host_capacity=100_000)
    ctx = gnm.Context(**cfg)
    ctx.load(reg)

    def read(w):
        return ctx.dense(w), ctx.rate_stats(w, hist=True), ctx.hosts(w)
    stream = gnm.Stream(ctx, budget_bytes=3 * 20_000 * 24, n_cuda_streams=3)
    done = _serve(gnm, stream, lambda a, b: gnm.Records.host({k: v[a:b] for k, v in pool.items()}),
                  wins, order, empty_close, read)
    stream.close()
    alone = gnm.Context(**cfg)
    alone.load(reg)
    for w, sl in wins.items():
        dense, rs, hosts = done[w][3]
        alone.process(gnm.Records.to_device(_concat(pool, sl)), w)
        for x, y in zip(dense, alone.dense(w)):
            np.testing.assert_array_equal(x, y)
        for x, y in zip(rs, alone.rate_stats(w, hist=True)):
            np.testing.assert_array_equal(x, y)
        for x, y in zip(hosts, alone.hosts(w)):
            np.testing.assert_array_equal(x, y)
    alone.close()
    ctx.close()


@pytest.mark.parametrize("pool_kind,host_records", [("pageable", "AUTO"), ("pinned", "AUTO"),
                                                    ("pinned", "STAGE"), ("pinned", "IN_PLACE")])
def test_submit_many_equals_alone(gnm, regs, pool_kind, host_records):
    """Batches given as slices of one pool in submit_many calls (closes among them) serve
    every window as when it is processed alone: a pageable pool is staged, a page-locked one
    is read in place unless the context stages host records."""
    reg = regs["c1"]
    rng = np.random.default_rng(23)
    pool = fg.make_records(reg, 200_000, seed=31)
    wins, order, empty_close = _plan_mix(rng, 8, 200_000, 20_000, empty_close_every=3)
    ev = []
    for w, j in order:
        a, b = wins[w][j]
        last = j == len(wins[w]) - 1
        ev.append((a, b - a, w, int(last and w not in empty_close)))
        if last and w in empty_close:
            ev.append((0, 0, w, 1))
    ctx = gnm.Context(window_slots=16, host_records=getattr(gnm, "HOST_" + host_records))
    ctx.load(reg)
    stream = gnm.Stream(ctx, budget_bytes=2 * 20_000 * 24, n_cuda_streams=3)
    hold = None
    if pool_kind == "pinned":
        hold, ppool = _pinned(pool)
        recs = gnm.Records(ppool)
    else:
        recs = gnm.Records.host(pool)
    done = {}
    for k in range(0, len(ev), 5):
        part = ev[k:k + 5]
        n = stream.submit_many(recs, [e[0] for e in part], [e[1] for e in part], [e[2] for e in part],
                               [e[3] for e in part])
        assert n == len(part)
        for wid, *_ in stream.poll():
            done[wid] = ctx.dense(wid)
    while len(done) < len(wins):
        for wid, *_ in stream.poll(wait_all=True):
            done[wid] = ctx.dense(wid)
    stream.close()
    alone = gnm.Context(window_slots=16)
    alone.load(reg)
    for w, sl in wins.items():
        alone.process(gnm.Records.to_device(_concat(pool, sl)), w)
        st_a, un_a, r_a, f_a = alone.dense(w)
        np.testing.assert_array_equal(done[w][0], st_a)
        np.testing.assert_array_equal(done[w][1], un_a)
        assert_rates_close(done[w][2], r_a)
        np.testing.assert_array_equal(done[w][3], f_a)
    alone.close()
    ctx.close()


def test_in_place_server_refuses_pageable_batches(gnm, regs):
    """A context that reads host records only in place refuses a pageable host batch (and a
    pool of them) and still serves page-locked ones."""
    reg = regs["c1"]
    pool = fg.make_records(reg, 50_000, seed=7)
    ctx = gnm.Context(window_slots=4, host_records=gnm.HOST_IN_PLACE)
    ctx.load(reg)
    stream = gnm.Stream(ctx, budget_bytes=1 << 24, n_cuda_streams=2)
    with pytest.raises(gnm.GnmError, match="INVAL"):
        stream.submit(gnm.Records.host(pool), 1, close=True)
    with pytest.raises(gnm.GnmError, match="INVAL"):
        stream.submit_many(gnm.Records.host(pool), [0], [10], [1], [1])
    hold, ppool = _pinned(pool)
    stream.submit(gnm.Records(ppool), 2, close=True)
    done = {wid for wid, *_ in stream.poll(wait_all=True)}
    assert done == {2}
    alone = gnm.Context(window_slots=4)
    alone.load(reg)
    alone.process(gnm.Records.to_device(pool), 2)
    for x, y in zip(ctx.dense(2), alone.dense(2)):
        np.testing.assert_array_equal(x, y)
    stream.close()
    alone.close()
    ctx.close()
