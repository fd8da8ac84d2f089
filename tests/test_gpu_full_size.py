"""Parity at the benchmark's full sizes, in the launch configurations bench.py times:
- 256 uneven windows, 84.5 M records, one autotuned CUDA-graph launch: sampled windows
  against the oracle one by one, and for every window the invariant that its sums over
  keys add up to its record count and octets;
- one 50 M-record window on the learned-index registry with the 4,096-leaf minimax model
  (window <= 64 proven): the whole window against the oracle;
- the same window with the sparse per-flow rate statistics: sampled keys' medians, least
  and greatest rates against the oracle;
- the 24-hour serving schedule (1,440 windows) through the streaming server: every 60th
  window and 10 random ones against the oracle.
Integers bit-exact, rates within 1e-12 (and bit-identical where compared directly)."""
import numpy as np
import pytest

import flowgen as fg
import oracle
from helpers import assert_window_matches, oracle_full

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gnm():
    from paper_1108_1785_gb300 import build, gnm as g
    build.build()
    return g


def test_batched_256_windows_full_size(gnm):
    reg = fg.registry_c1()
    counts = fg.uneven_windows_c4()
    rec, off = fg.batched_records_c4(reg, counts)
    n_win = len(off) - 1
    assert n_win == 256 and int(off[-1]) > 80_000_000
    ctx = gnm.Context(window_slots=n_win + 8)
    ctx.load(reg)
    d = gnm.Records.to_device(rec)
    ids = np.arange(n_win, dtype=np.uint64)
    ctx.autotune(d, off, ids)
    plan = ctx.plan(d, off, ids)
    plan.launch()
    torch.cuda.synchronize()
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    rng = np.random.default_rng(4)
    sample = sorted({int(np.argmax(counts)), int(np.argmin(counts)), 0, n_win - 1,
                     *rng.choice(n_win, size=6, replace=False).tolist()})
    for w in sample:
        part = {k: v[off[w]:off[w + 1]] for k, v in rec.items()}
        assert_window_matches(ctx.dense(int(ids[w])), oracle_full(reg, part, lpm=lpm))
    for w in range(n_win):  # every record lands in one key; octets add up
        st, un, _, _ = ctx.dense(int(ids[w]))
        assert int(st[:, 0].sum()) + int(un[:, 0].sum()) == int(counts[w])
        o = rec["dOctets"][off[w]:off[w + 1]].astype(np.uint64).sum()
        assert int(st[:, 1].sum()) + int(un[:, 1].sum()) == int(o)
    plan.close()
    ctx.close()


def test_learned_index_window_full_size(gnm):
    reg = fg.registry_c3()
    n = 50_000_000
    rec = fg.make_records(reg, n, seed=2, p_reg=0.9, zipf_s=0.9)
    keys = torch.from_numpy(fg.lookup_keys_c3(reg, 10_000_000).view(np.int32)).cuda()
    ctx = gnm.Context(window_slots=4, lookup_mode=gnm.LOOKUP_RMI)
    ctx.load(reg)
    rep = ctx.rmi_train(keys, root_kind=gnm.ROOT_LINEAR, n_leaves=4096, leaf_iters=4)
    assert rep.eps_max <= 64
    ctx.rmi_violations(reset=True)
    plan = ctx.plan(gnm.Records.to_device(rec), [0, n], [1])
    plan.launch()
    torch.cuda.synchronize()
    got = ctx.dense(1)
    want = oracle_full(reg, rec, n_threads=16)
    assert_window_matches(got, want)
    gr, wr = np.asarray(got[2]), np.asarray(want[2])
    ok = ~np.isnan(wr)
    np.testing.assert_array_equal(gr[ok].view(np.uint64), wr[ok].view(np.uint64))
    assert ctx.rmi_violations() == 0
    plan.close()
    ctx.close()


def test_learned_index_window_sparse_rate_stats_full_size(gnm):
    """Per-flow rate statistics on the 100,000-site registry (200,004 keys: dense histograms
    would take 8 GB per window), one window of 50,000,000 records through the learned index
    with the sparse log: medians, least and greatest rates equal the oracle's on 300 sampled
    keys (the busiest, random ones and any without eligible flows), and the log's cells add
    up to every key's eligible flows."""
    reg = fg.registry_c3()
    n = 50_000_000
    rec = fg.make_records(reg, n, seed=2, p_reg=0.9, zipf_s=0.9)
    keys = torch.from_numpy(fg.lookup_keys_c3(reg, 10_000_000).view(np.int32)).cuda()
    ctx = gnm.Context(window_slots=2, lookup_mode=gnm.LOOKUP_RMI, rate_stats=2)
    ctx.load(reg)
    ctx.rmi_train(keys, root_kind=gnm.ROOT_LINEAR, n_leaves=4096, leaf_iters=4)
    plan = ctx.plan(gnm.Records.to_device(rec), [0, n], [1])
    plan.launch()
    torch.cuda.synchronize()
    rmin, rmax, med, _ = ctx.rate_stats(1)
    st, _, _, _ = ctx.dense(1)
    ck, cb, cc = ctx.rate_cells(1)
    efl = np.bincount(ck, weights=cc, minlength=2 * reg.n_sites).astype(np.uint64)
    np.testing.assert_array_equal(efl, st[:, 3])  # e_flows per key
    rng = np.random.default_rng(9)
    busy = np.argsort(st[:, 3])[-50:]
    some = rng.choice(np.nonzero(st[:, 3])[0], 230, replace=False)
    zero = np.nonzero(st[:, 3] == 0)[0]  # (at this size every key may have eligible flows)
    empty = rng.choice(zero, min(20, zero.size), replace=False)
    sample = np.unique(np.concatenate([busy, some, empty]))
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    lo, hi, m, cnt = oracle.rate_stats_keys(lpm, reg.local_prefix, reg.local_len, reg.n_sites, rec, sample)
    np.testing.assert_array_equal(cnt, st[sample, 3])
    np.testing.assert_array_equal(med[sample], m)
    np.testing.assert_array_equal(rmin[sample], lo)
    np.testing.assert_array_equal(rmax[sample], hi)
    plan.close()
    ctx.close()


def test_served_day_checked_windows_full_size(gnm):
    """The 24-hour serving schedule at full size (1,440 one-minute windows, 86.4e9 records in
    Poisson batches of 1,000-500,000 records cut from a pinned 20,000,000-record pool) through
    the streaming server with the 4,096-leaf learned index, submitted as fast as the 4 GB
    budget admits: every 60th window and 10 random ones equal the oracle (sums, unmatched
    classes and flags bit-exact, rates within 1e-12), and every window's record count is
    the schedule's."""
    reg = fg.registry_c3()
    pool_n = 20_000_000
    pool = fg.make_records(reg, pool_n, seed=4, p_reg=0.9, zipf_s=0.9)
    pinned = {k: torch.from_numpy(np.ascontiguousarray(pool[k]).view(np.int32)).pin_memory() for k in gnm.FIELDS}
    hpool = {k: v.numpy().view(np.uint32) for k, v in pinned.items()}
    t, sz = fg.serving_schedule_c5(hours=24.0)
    rng = np.random.default_rng(5)
    offs = rng.integers(0, pool_n - sz + 1)
    win = (t // 60.0).astype(np.int64)
    n_win = 24 * 60
    checked = sorted(set(range(0, n_win, 60)) | set(rng.choice(n_win, 10, replace=False).tolist()))
    assert len(checked) == 34
    ctx = gnm.Context(window_slots=16)
    ctx.load(reg)
    ctx.rmi_train(torch.from_numpy(fg.lookup_keys_c3(reg, 10_000_000).view(np.int32)).cuda(), n_leaves=4096)
    ev_b, ev_c, ev_w, ev_f = [], [], [], []
    bi = 0
    for w in range(n_win):  # batches of minute w, then its close
        while bi < t.size and win[bi] == w:
            ev_b.append(int(offs[bi])), ev_c.append(int(sz[bi])), ev_w.append(w), ev_f.append(0)
            bi += 1
        ev_b.append(0), ev_c.append(0), ev_w.append(w), ev_f.append(1)
    got, records = {}, {}

    def take(reports):
        for r in reports:
            assert r[3] == 0
            records[r[0]] = r[1]
            if r[0] in checked:
                got[r[0]] = ctx.dense(r[0])

    with gnm.Stream(ctx, budget_bytes=4 << 30, n_cuda_streams=4) as srv:
        pool_recs = gnm.Records(hpool)
        for k in range(0, len(ev_b), 512):
            srv.submit_many(pool_recs, ev_b[k:k + 512], ev_c[k:k + 512], ev_w[k:k + 512], ev_f[k:k + 512])
            take(srv.poll())
        take(srv.poll(wait_all=True))
    assert sorted(records) == list(range(n_win))
    np.testing.assert_array_equal([records[w] for w in range(n_win)], np.bincount(win, weights=sz, minlength=n_win))
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    for w in checked:
        idx = np.nonzero(win == w)[0]
        rec = {k: np.concatenate([pool[k][offs[i]:offs[i] + sz[i]] for i in idx]) for k in gnm.FIELDS}
        assert_window_matches(got[w], oracle_full(reg, rec, lpm=lpm, n_threads=16))
    ctx.close()
