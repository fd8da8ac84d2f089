"""Batched plans (CUDA graph over many uneven windows) and the autotuner: every window
of the batch equals the oracle, on every replay and after tuning."""
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


@pytest.fixture(scope="module")
def batch():
    reg = fg.registry_c1()
    counts = fg.uneven_windows_c4(n_windows=48, seed=9, lo=1000, hi=200_000, median=20_000)
    counts[5] = 0  # an empty window in the middle
    rec, off = fg.batched_records_c4(reg, counts, seed=9)
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    expect = [oracle_full(reg, {k: v[off[w]:off[w + 1]] for k, v in rec.items()}, lpm=lpm)
              for w in range(len(counts))]
    return reg, rec, off, expect


def test_plan_replays_match_oracle(gnm, batch):
    reg, rec, off, expect = batch
    ctx = gnm.Context(window_slots=64)
    ctx.load(reg)
    d = gnm.Records.to_device(rec)
    ids = np.arange(len(off) - 1) + 1000
    plan = ctx.plan(d, off, ids)
    for rep in range(3):
        plan.launch()
        assert ctx.last_launch_count() == 1  # shared-memory registry: one fused kernel
        for w in range(len(ids)):
            assert_window_matches(ctx.dense(int(ids[w])), expect[w])
    with pytest.raises(gnm.GnmError, match="plan"):
        ctx.process(d, int(ids[0]))  # a plan's window id cannot be reused elsewhere
    plan.close()
    ctx.process(gnm.Records({k: v[:10] for k, v in d.fields.items()}), int(ids[0]))  # released with the plan
    ctx.close()


def test_plan_sees_new_buffer_contents(gnm, batch):
    """Plans bind buffers, not contents: refill the buffers and replay."""
    reg, rec, off, expect = batch
    ctx = gnm.Context(window_slots=64)
    ctx.load(reg)
    d = gnm.Records.to_device(rec)
    ids = np.arange(len(off) - 1)
    plan = ctx.plan(d, off, ids)
    plan.launch()
    rec2, _ = fg.batched_records_c4(reg, np.diff(off), seed=10)
    for k in gnm.FIELDS:
        d.fields[k].copy_(torch.from_numpy(rec2[k].view(np.int32)))
    plan.launch()
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    for w in (0, 7, 20, 47):
        host = {k: v[off[w]:off[w + 1]] for k, v in rec2.items()}
        assert_window_matches(ctx.dense(int(ids[w])), oracle_full(reg, host, lpm=lpm))
    plan.close()
    ctx.close()


def test_autotune_then_exact(gnm, batch):
    reg, rec, off, expect = batch
    ctx = gnm.Context(window_slots=64)
    ctx.load(reg)
    d = gnm.Records.to_device(rec)
    ids = np.arange(len(off) - 1) + 5
    rep = ctx.autotune(d, off, ids)
    assert rep.n_tried >= 8
    assert 0 < rep.best_ms <= rep.default_ms * 1.05
    assert rep.block_threads in (256, 512, 768, 1024) and rep.unroll in (1, 2, 3)
    for w in range(len(ids)):
        assert_window_matches(ctx.dense(int(ids[w])), expect[w])
    ctx.process_windows(d, off, ids)  # tuned shape from now on
    for w in range(len(ids)):
        assert_window_matches(ctx.dense(int(ids[w])), expect[w])
    ctx.close()


def test_windows_results_batch_readout(gnm, batch):
    reg, rec, off, expect = batch
    ctx = gnm.Context(window_slots=64)
    ctx.load(reg)
    ids = np.arange(len(off) - 1) + 77
    ctx.process_windows(gnm.Records.to_device(rec), off, ids)
    nk = 2 * reg.n_sites
    W = len(ids)
    st = np.empty((W, nk, 6), np.uint64)
    un = np.empty((W, 4, 3), np.uint64)
    r = np.empty((W, nk), np.float64)
    f = np.empty((W, nk), np.uint8)
    ctx.windows_results(ids, st, un, r, f)
    for w in range(W):
        assert_window_matches((st[w], un[w], r[w], f[w]), expect[w])
    # any order and subset (runs of consecutive result slots are read with one copy each)
    perm = np.concatenate([np.random.default_rng(2).permutation(W)[:20], np.arange(30, 40)])
    st2, un2 = np.empty((perm.size, nk, 6), np.uint64), np.empty((perm.size, 4, 3), np.uint64)
    r2, f2 = np.empty((perm.size, nk), np.float64), np.empty((perm.size, nk), np.uint8)
    ctx.windows_results(ids[perm], st2, un2, r2, f2)
    for j, w in enumerate(perm):
        assert_window_matches((st2[j], un2[j], r2[j], f2[j]), expect[w])
    ctx.close()


def test_windows_results_async_overlaps_processing(gnm, batch):
    """Asynchronous readouts on a second stream while the other set of windows is processed:
    two sets of window ids, each reprocessed with a different batch (the windows in reverse
    order) while the copy of its previous results may still run. Every copy holds the
    results of the batch processed just before it (the reprocessing waits for the copy)."""
    reg, rec, off, expect = batch
    W = len(off) - 1
    # the same windows in reverse order
    order = np.arange(W)[::-1]
    rec_r = {k: np.concatenate([v[off[w]:off[w + 1]] for w in order]) for k, v in rec.items()}
    off_r = np.concatenate([[0], np.cumsum([off[w + 1] - off[w] for w in order])]).astype(np.int64)
    batches = [(rec, off, expect), (rec_r, off_r, [expect[w] for w in order])]
    dev = [gnm.Records.to_device(b[0]) for b in batches]
    ctx = gnm.Context(window_slots=2 * W + 4)
    ctx.load(reg)
    nk = 2 * reg.n_sites
    sets = [np.arange(W) + 5000, np.arange(W) + 6000]
    proc, copy = torch.cuda.Stream(), torch.cuda.Stream()

    def pinned(shape, dt):
        t = torch.empty(int(np.prod(shape)) * np.dtype(dt).itemsize, dtype=torch.uint8).pin_memory()
        return t.numpy().view(dt).reshape(shape)

    steps = 6
    outs = [(pinned((W, nk, 6), np.uint64), pinned((W, 4, 6), np.uint64), pinned((W, nk), np.float64),
             pinned((W, nk), np.uint8)) for _ in range(steps)]
    for k in range(steps):
        b = (k // 2) % 2  # set k % 2 gets batch 0, 0, 1, 1, 0, 0 ...: each set alternates
        ctx.process_windows(dev[b], batches[b][1], sets[k % 2], proc)
        ctx.windows_results_async(sets[k % 2], *outs[k], stream=copy)
    copy.synchronize()
    proc.synchronize()
    for k in range(steps):
        b = (k // 2) % 2
        st, un6, r, f = outs[k]
        for w in range(W):
            assert_window_matches((st[w], un6[w][:, :3], r[w], f[w]), batches[b][2][w])
    ctx.close()


@pytest.mark.parametrize("which", ["c1", "c2"])
def test_plan_kernel_times(gnm, which):
    """A plan made with kernel timing names its kernels in launch order, each with a positive
    device duration, and still gives the oracle's results; without the flag it refuses."""
    reg = fg.registry_c1() if which == "c1" else fg.registry_c2()
    rec = fg.make_records(reg, 400_000, seed=31)
    off = [0, 150_000, 150_000, 400_000]
    ctx = gnm.Context(window_slots=8)
    ctx.load(reg)
    d = gnm.Records.to_device(rec)
    plain = ctx.plan(d, off, [1, 2, 3])
    plain.launch()
    with pytest.raises(gnm.GnmError, match="STATE"):
        plain.kernel_times()
    plain.close()
    plan = ctx.plan(d, off, [1, 2, 3], kernel_times=True)
    with pytest.raises(gnm.GnmError, match="STATE"):
        plan.kernel_times()  # not launched yet
    for _ in range(2):
        plan.launch()
        kt = plan.kernel_times()
        names = [k for k, _ in kt]
        if which == "c1":  # registry in shared memory: one fused kernel
            assert names == ["k_aggregate"]
        else:
            assert names == ["k_keys", "k_aggregate", "k_finalize_windows"]
        assert all(ms > 0 for _, ms in kt)
    for w, (a, b) in zip([1, 2, 3], zip(off[:-1], off[1:])):
        assert_window_matches(ctx.dense(w), oracle_full(reg, {k: v[a:b] for k, v in rec.items()}))
    plan.close()
    ctx.close()
