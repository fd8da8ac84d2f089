"""The learned index on the GPU: training gradients against the FP64 oracle, trained
stages against closed-form least squares, error bounds against the oracle's endpoint
analysis, lookups bit-exact against the oracle (with and without proven bounds), and
what the model gains over the plain binary search."""
import numpy as np
import pytest

import flowgen as fg
import oracle
from helpers import assert_window_matches, oracle_full
from oracle import rmi_ref

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gnm():
    from paper_1108_1785_gb300 import build, gnm as g
    build.build()
    return g


def remote_of(reg, rec):
    src = rec["srcaddr"].astype(np.int64)
    loc = np.zeros(src.shape, bool)
    for p, l in zip(reg.local_prefix, reg.local_len):
        loc |= (src >> (32 - int(l))) == (int(p) >> (32 - int(l)))
    return np.where(loc, rec["dstaddr"], rec["srcaddr"]).astype(np.uint32)


@pytest.fixture(scope="module")
def c3():
    reg = fg.registry_c3()
    lpm = oracle.LPM(reg.prefix, reg.plen, reg.site)
    starts, sites = lpm.flatten()
    rec = fg.make_records(reg, 2_000_000, seed=21, p_reg=0.9, zipf_s=0.9)
    keys = remote_of(reg, rec)
    return reg, lpm, starts, sites, rec, keys


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def probe_set(starts, n_random=500_000, seed=0):
    s = starts.astype(np.int64)
    x = np.concatenate([s, s - 1, s + 1, [0, 0xFFFFFFFF], np.random.default_rng(seed).integers(0, 1 << 32, n_random)])
    return x[(x >= 0) & (x < (1 << 32))].astype(np.uint32)


def test_linear_gradient_matches_fp64(gnm):
    ctx = gnm.Context()
    rng = np.random.default_rng(4)
    z = rng.normal(size=300_000).astype(np.float32)
    y = (3 * z + 0.5 + rng.normal(size=z.size)).astype(np.float32)
    for w, c in [(0.0, 0.0), (2.5, -1.0), (3.0, 0.5)]:
        g = ctx.rmi_linear_grad(torch.from_numpy(z).cuda(), torch.from_numpy(y).cuda(), w, c)
        loss, gw, gc = rmi_ref.linear_grad(np.float32(w), np.float32(c), z, y)
        scale = max(abs(gw), abs(gc), 1e-3)
        assert abs(g[0] - gw) <= 1e-4 * scale and abs(g[1] - gc) <= 1e-4 * scale
        assert g[2] == pytest.approx(loss, rel=1e-4)
    ctx.close()


@pytest.mark.parametrize("H", [8, 32])
def test_mlp_gradient_matches_fp64(gnm, H):
    ctx = gnm.Context()
    rng = np.random.default_rng(5 + H)
    p = {"w1": rng.normal(size=H), "b1": rng.normal(size=H) * 0.3, "w2": rng.normal(size=H), "b2": 0.1}
    flat = np.concatenate([p["w1"], p["b1"], p["w2"], [p["b2"]]]).astype(np.float32)
    p32 = {"w1": flat[:H].astype(np.float64), "b1": flat[H:2 * H].astype(np.float64),
           "w2": flat[2 * H:3 * H].astype(np.float64), "b2": float(flat[3 * H])}
    xn = rng.random(200_000).astype(np.float32)
    y = np.sqrt(xn).astype(np.float32)
    g = ctx.rmi_mlp_grad(torch.from_numpy(xn).cuda(), torch.from_numpy(y).cuda(), H, flat)
    loss, ref = rmi_ref.mlp_loss_grad(p32, xn.astype(np.float64), y.astype(np.float64))
    want = np.concatenate([ref["w1"], ref["b1"], ref["w2"], [ref["b2"]]])
    scale = np.max(np.abs(want))
    np.testing.assert_allclose(g[:3 * H + 1], want, rtol=1e-4, atol=1e-4 * scale)
    assert g[3 * H + 1] == pytest.approx(loss, rel=1e-4)
    ctx.close()


@pytest.fixture(scope="module")
def trained_linear(gnm, c3):
    """The learned-index workload's model: linear root, 4,096 minimax leaves, leaves whose
    window would exceed 64 split (the defaults)."""
    reg, lpm, starts, sites, rec, keys = c3
    ctx = gnm.Context(window_slots=4)
    ctx.load(reg)
    rep = ctx.rmi_train(to_dev(keys), root_kind=gnm.ROOT_LINEAR, n_leaves=4096, leaf_iters=4)
    return ctx, rep


@pytest.fixture(scope="module")
def trained_mse(gnm, c3):
    reg, lpm, starts, sites, rec, keys = c3
    ctx = gnm.Context(window_slots=2)
    ctx.load(reg)
    rep = ctx.rmi_train(to_dev(keys), root_kind=gnm.ROOT_LINEAR, n_leaves=4096, leaf_iters=4,
                        leaf_fit=gnm.FIT_MSE)
    return ctx, rep


def test_linear_rmi_bounds_equal_endpoint_analysis(gnm, c3, trained_linear):
    """The exhaustive GPU sweep's per-model bounds equal the oracle's endpoint analysis of
    the exported model (split leaves included), and meet the 4,096-leaf model's target:
    window eps_lo + eps_hi <= 64, so every |predicted - true position| <= 64."""
    reg, lpm, starts, sites, rec, keys = c3
    ctx, rep = trained_linear
    m = ctx.rmi_export()
    assert m["root_kind"] == gnm.ROOT_LINEAR and m["n_leaves"] == 4096
    assert m["n_models"] == rep.n_models == 4096 + int(sum((w >> 8) + 1 for w in m["split"] if w))
    assert rep.split_leaves == int(np.count_nonzero(m["split"]))
    elo, ehi = rmi_ref.eps_endpoints_models(starts, float(m["root"][0]), float(m["root"][1]), 4096, m["split"],
                                            m["a"], m["b"], m["x0"])
    np.testing.assert_array_equal(m["eps_lo"], elo)
    np.testing.assert_array_equal(m["eps_hi"], ehi)
    assert rep.eps_max == int(np.max(elo + ehi))
    assert rep.err_max == int(np.max(np.maximum(elo, ehi)))
    assert rep.eps_max <= 64 and rep.err_max <= 64
    print(f"\nlinear RMI: ranges {starts.size}, models {rep.n_models} ({rep.split_leaves} split leaves), "
          f"eps_max {rep.eps_max}, err_max {rep.err_max}, mean window {rep.eps_mean:.1f}, "
          f"train {rep.train_ms:.1f} ms, sweep {rep.sweep_ms:.1f} ms, empty leaves {rep.empty_leaves}")


def test_minimax_leaves_near_optimal(gnm, c3, trained_linear):
    """Every sampled model's proven error is within rounding of the FP64 optimum of the
    oracle's minimax fit over the same address interval."""
    reg, lpm, starts, sites, rec, keys = c3
    ctx, _ = trained_linear
    m = ctx.rmi_export()
    first, mlo, mhi = rmi_ref.split_tables(float(m["root"][0]), float(m["root"][1]), 4096, m["split"])
    models = [i for i in range(m["n_models"]) if not (i < 4096 and m["split"][i])]
    rng = np.random.default_rng(3)
    pick = sorted(set(rng.choice(models, size=150, replace=False).tolist()) |
                  set(np.argsort(np.maximum(m["eps_lo"], m["eps_hi"]))[-20:].tolist()))
    for i in pick:
        if i < 4096 and m["split"][i]:
            continue
        np.testing.assert_equal(int(m["x0"][i]), int(min(mlo[i], (1 << 32) - 1)))
        E = rmi_ref.fit_interval_minimax(starts, int(mlo[i]), int(mhi[i]))[2]
        got = max(int(m["eps_lo"][i]), int(m["eps_hi"][i]))
        assert got <= np.ceil(E + 0.5) + 2, f"model {i}: bound {got}, optimum {E:.2f}"


def test_minimax_training_is_deterministic(gnm, c3):
    """Two trainings on the same keys give the same model bit for bit (ordered reductions)."""
    reg, lpm, starts, sites, rec, keys = c3
    out = []
    for _ in range(2):
        ctx = gnm.Context(window_slots=1)
        ctx.load(reg)
        rep = ctx.rmi_train(to_dev(keys[:500_000]), n_leaves=2048)
        out.append((ctx.rmi_export(), rep.eps_max, rep.leaf_loss))
        ctx.close()
    (m1, e1, l1), (m2, e2, l2) = out
    assert e1 == e2 and l1 == l2
    for k in ("root", "split", "a", "b", "x0", "eps_lo", "eps_hi"):
        np.testing.assert_array_equal(m1[k].view(np.uint32), m2[k].view(np.uint32), err_msg=k)


def test_minimax_beats_mse_on_the_bound(gnm, trained_linear, trained_mse):
    """What the minimax fit gains over the mean-squared-error leaves on the same root: a far
    smaller proven bound, and a smaller mean window over the training lookups."""
    _, rep = trained_linear
    _, mse = trained_mse
    assert mse.n_models == 4096 and mse.split_leaves == 0
    assert rep.eps_max < mse.eps_max / 2
    assert rep.eps_mean < mse.eps_mean
    print(f"\nminimax leaves: eps_max {rep.eps_max}, mean window {rep.eps_mean:.1f}; "
          f"MSE leaves: eps_max {mse.eps_max}, mean window {mse.eps_mean:.1f}")


def test_linear_rmi_leaves_are_least_squares(gnm, c3, trained_mse):
    reg, lpm, starts, sites, rec, keys = c3
    ctx, _ = trained_mse
    m = ctx.rmi_export()
    pos = np.searchsorted(starts, keys, side="right") - 1
    leaf = rmi_ref.root_linear(float(m["root"][0]), float(m["root"][1]), keys, 4096)
    checked = 0
    for l in np.unique(leaf)[:: max(1, len(np.unique(leaf)) // 40)]:
        sel = leaf == l
        if sel.sum() < 50:
            continue
        d = (keys[sel].astype(np.int64) - int(m["x0"][l])).astype(np.float32).astype(np.float64)
        y = pos[sel].astype(np.float64)
        if np.ptp(d) == 0:
            continue
        a, b = rmi_ref.lstsq_line(d, y)
        a = max(a, 0.0)
        got = float(m["a"][l]) * d + float(m["b"][l])
        ls = a * d + b
        assert np.max(np.abs(got - ls)) <= 1e-3 * max(1.0, np.ptp(y)) + 0.05, f"leaf {l}"
        checked += 1
    assert checked >= 20


def test_linear_rmi_lookups_exact_without_fallback(gnm, c3, trained_linear):
    reg, lpm, starts, sites, rec, keys = c3
    ctx, _ = trained_linear
    ctx.rmi_violations(reset=True)
    x = probe_set(starts)
    dx = to_dev(x)
    site = torch.empty_like(dx)
    pos = torch.empty_like(dx)
    ctx.lookup(dx, site, pos)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(pos.cpu().numpy().view(np.uint32), np.searchsorted(starts, x, side="right") - 1)
    np.testing.assert_array_equal(site.cpu().numpy().view(np.uint32), lpm.lookup(x))
    assert ctx.rmi_violations() == 0  # exhaustive bounds hold for every address


def test_rmi_window_equals_bsearch_and_oracle(gnm, c3, trained_linear):
    reg, lpm, starts, sites, rec, keys = c3
    ctx, _ = trained_linear
    d = gnm.Records.to_device(rec)
    ctx.process(d, 1)  # AUTO lookup: learned index
    expect = oracle_full(reg, rec, lpm=lpm)
    assert_window_matches(ctx.dense(1), expect)
    for mode in (gnm.LOOKUP_BSEARCH, gnm.LOOKUP_RADIX):
        plain = gnm.Context(window_slots=2, lookup_mode=mode)
        plain.load(reg)
        plain.process(d, 1)
        assert_window_matches(plain.dense(1), expect)
        plain.close()


def test_rmi_gain_over_binary_search(gnm, c3, trained_linear):
    """Same GPU, same addresses: the model's window needs fewer dependent probes than
    the full search, and the lookup kernel is faster."""
    reg, lpm, starts, sites, rec, keys = c3
    ctx, rep = trained_linear
    plain = gnm.Context(lookup_mode=gnm.LOOKUP_BSEARCH)
    plain.load(reg)
    n = 20_000_000
    x = np.resize(keys, n)
    dx = to_dev(x)
    s1 = torch.empty_like(dx)
    s2 = torch.empty_like(dx)

    def t(c, out):
        for _ in range(2):
            c.lookup(dx, out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(5):
            c.lookup(dx, out)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 5

    tb, tr = t(plain, s1), t(ctx, s2)
    assert torch.equal(s1, s2)
    radix = gnm.Context(lookup_mode=gnm.LOOKUP_RADIX)
    radix.load(reg)
    s3 = torch.empty_like(dx)
    td = t(radix, s3)
    assert torch.equal(s1, s3)
    radix.close()
    print(f"\nradix-directed lookups: {td:.3f} ms")
    probes_plain = np.ceil(np.log2(starts.size))
    probes_rmi = np.log2(rep.eps_mean + 1) + 1
    print(f"\nlookups of {n:,} addresses: bsearch {tb:.3f} ms, learned index {tr:.3f} ms "
          f"({tb / tr:.2f}x); probes {probes_plain:.0f} vs ~{probes_rmi:.1f}")
    assert probes_rmi < probes_plain / 2
    assert tr < tb
    plain.close()


def test_rmi_sample_bounds_fall_back_exactly(gnm, c3):
    """Bounds from a small training sample only: lookups outside it may miss the model
    window; the fallback keeps every result exact and counts the misses."""
    reg, lpm, starts, sites, rec, keys = c3
    ctx = gnm.Context(window_slots=2)
    ctx.load(reg)
    ctx.rmi_train(to_dev(keys[:20000]), n_leaves=4096, exhaustive_eps=0, leaf_fit=gnm.FIT_MSE)
    ctx.rmi_violations(reset=True)
    x = probe_set(starts, seed=1)
    dx = to_dev(x)
    site = torch.empty_like(dx)
    ctx.lookup(dx, site)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(site.cpu().numpy().view(np.uint32), lpm.lookup(x))
    assert ctx.rmi_violations() > 0
    ctx.close()


@pytest.mark.parametrize("split", ["SPLIT_TWO_KERNELS", "SPLIT_FUSED"])
@pytest.mark.parametrize("unroll", [1, 2])
def test_rmi_window_fallback_exact(gnm, c3, split, unroll):
    """The window kernels' learned-index lookups (several in lock step per thread) with
    bounds from a small sample: records whose address misses its model window take the full
    search, the window stays equal to the oracle, and the misses are counted."""
    reg, lpm, starts, sites, rec, keys = c3
    ctx = gnm.Context(window_slots=2, split=getattr(gnm, split), unroll=unroll)
    ctx.load(reg)
    ctx.rmi_train(to_dev(keys[:20000]), n_leaves=4096, exhaustive_eps=0, leaf_fit=gnm.FIT_MSE)
    assert ctx.registry_info().lookup_mode == gnm.LOOKUP_RMI
    ctx.rmi_violations(reset=True)
    rng = np.random.default_rng(4)
    w = {k: v[:300_001] for k, v in rec.items()}
    w["srcaddr"] = w["srcaddr"].copy()
    w["dstaddr"] = w["dstaddr"].copy()
    # uniformly random remote addresses in a third of the records: many fall outside the
    # sampled key range of their leaves
    sel = rng.random(w["srcaddr"].size) < 0.33
    lp, ll = int(reg.local_prefix[0]), int(reg.local_len[0])
    w["srcaddr"][sel] = rng.integers(0, 1 << 32, int(sel.sum()), dtype=np.uint64).astype(np.uint32)
    w["dstaddr"][sel] = (lp | rng.integers(0, 1 << (32 - ll), int(sel.sum()))).astype(np.uint32)
    ctx.process(gnm.Records.to_device(w), 1)
    assert_window_matches(ctx.dense(1), oracle_full(reg, w, lpm=lpm))
    assert ctx.rmi_violations() > 0
    ctx.close()


@pytest.mark.parametrize("table", ["PARTITION", "HASH"])
def test_large_key_space_windows(gnm, c3, table):
    """200,004 keys (100,000 sites): three uneven windows in one launch, with the records
    regrouped by (window, key group) before the aggregation (20 groups per window) or with
    the per-CTA hash cache; every window equals the oracle."""
    reg, lpm, starts, sites, rec, keys = c3
    ctx = gnm.Context(window_slots=4, table_mode=getattr(gnm, "TABLE_" + table))
    ctx.load(reg)
    off = [0, 1, 700_001, 2_000_000]
    d = gnm.Records.to_device(rec)
    plan = ctx.plan(d, off, [7, 8, 9], kernel_times=True)
    plan.launch()
    names = [k for k, _ in plan.kernel_times()]
    if table == "PARTITION":  # (the key kernel also counts the records of every bucket)
        assert names == ["k_keys", "k_part_scan", "k_part_scatter", "k_aggregate", "k_finalize_windows"]
    else:
        assert names == ["k_keys", "k_aggregate", "k_finalize_windows"]
    for w, (a, b) in zip([7, 8, 9], zip(off[:-1], off[1:])):
        assert_window_matches(ctx.dense(w), oracle_full(reg, {k: v[a:b] for k, v in rec.items()}, lpm=lpm))
    plan.close()
    ctx.close()


def test_mlp_root_rmi_exact(gnm, c3):
    reg, lpm, starts, sites, rec, keys = c3
    ctx = gnm.Context(window_slots=2)
    ctx.load(reg)
    rep = ctx.rmi_train(to_dev(keys), root_kind=gnm.ROOT_MLP, hidden=32, mlp_steps=300, n_leaves=4096)
    assert np.isfinite(rep.root_loss) and rep.root_loss < (4096 ** 2) / 12  # beats a constant root
    ctx.rmi_violations(reset=True)
    x = probe_set(starts, n_random=200_000, seed=2)
    dx = to_dev(x)
    site = torch.empty_like(dx)
    ctx.lookup(dx, site)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(site.cpu().numpy().view(np.uint32), lpm.lookup(x))
    assert ctx.rmi_violations() == 0
    print(f"\nMLP-root RMI: root mse {rep.root_loss:.2f} (leaf units), eps_max {rep.eps_max}, "
          f"mean window {rep.eps_mean:.1f}, train {rep.train_ms:.1f} ms, sweep {rep.sweep_ms:.1f} ms")
    ctx.close()


def test_mlp_root_window_exact(gnm, c3):
    """The MLP-root model inside the window kernels (key kernel, regrouping, aggregation):
    two windows equal the oracle and no lookup leaves its proven window."""
    reg, lpm, starts, sites, rec, keys = c3
    ctx = gnm.Context(window_slots=4)
    ctx.load(reg)
    ctx.rmi_train(to_dev(keys), root_kind=gnm.ROOT_MLP, hidden=16, mlp_steps=200, n_leaves=2048)
    assert ctx.registry_info().lookup_mode == gnm.LOOKUP_RMI
    ctx.rmi_violations(reset=True)
    off = [0, 123_457, 400_000]
    ctx.process_windows(gnm.Records.to_device({k: v[:400_000] for k, v in rec.items()}), off, [1, 2])
    for w, (a, b) in zip([1, 2], zip(off[:-1], off[1:])):
        assert_window_matches(ctx.dense(w), oracle_full(reg, {k: v[a:b] for k, v in rec.items()}, lpm=lpm))
    assert ctx.rmi_violations() == 0
    ctx.close()


def test_rmi_export_import_roundtrip(gnm, c3, trained_linear):
    reg, lpm, starts, sites, rec, keys = c3
    ctx, _ = trained_linear
    m = ctx.rmi_export()
    other = gnm.Context()
    other.load(reg)
    assert np.count_nonzero(m["split"]) > 0
    other.rmi_import(m["root_kind"], m["root"], m["a"], m["b"], m["x0"], split=m["split"])
    m2 = other.rmi_export()
    for k in ("split", "a", "b", "x0", "eps_lo", "eps_hi"):
        np.testing.assert_array_equal(m[k], m2[k])
    # a split table that does not add up to the model count is refused
    bad = m["split"].copy()
    bad[np.nonzero(bad)[0][0]] += 1 << 8
    with pytest.raises(gnm.GnmError, match="add up"):
        other.rmi_import(m["root_kind"], m["root"], m["a"], m["b"], m["x0"], split=bad)
    other.close()


@pytest.mark.parametrize("leaves,placement,split", [(4096, "L2", "TWO_KERNELS"), (4096, "L2", "FUSED"),
                                                    (65536, "AUTO", "TWO_KERNELS")])
def test_rmi_leaves_in_global_memory(gnm, c3, trained_linear, leaves, placement, split):
    """Leaf parameters read from global memory, one interleaved 16-byte load per lookup: asked
    for with the L2 placement, and automatic for 65,536 leaves (1 MB, beyond shared memory).
    Batch lookups and windows are exact, with no fallback; more leaves give tighter bounds."""
    reg, lpm, starts, sites, rec, keys = c3
    ctx = gnm.Context(window_slots=4, placement=getattr(gnm, "PLACE_" + placement),
                      split=getattr(gnm, "SPLIT_" + split))
    ctx.load(reg)
    rep = ctx.rmi_train(to_dev(keys), root_kind=gnm.ROOT_LINEAR, n_leaves=leaves, leaf_iters=4)
    if leaves == 65536:  # tighter than the 4,096-leaf model trained on the same keys
        assert rep.eps_mean < trained_linear[1].eps_mean
    ctx.rmi_violations(reset=True)
    x = probe_set(starts, n_random=200_000)
    dx = to_dev(x)
    site = torch.empty_like(dx)
    pos = torch.empty_like(dx)
    ctx.lookup(dx, site, pos)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(pos.cpu().numpy().view(np.uint32), np.searchsorted(starts, x, side="right") - 1)
    np.testing.assert_array_equal(site.cpu().numpy().view(np.uint32), lpm.lookup(x))
    ctx.process(gnm.Records.to_device(rec), 1)
    assert_window_matches(ctx.dense(1), oracle_full(reg, rec, lpm=lpm))
    assert ctx.rmi_violations() == 0
    ctx.close()


def test_rmi_leaves_too_large_for_shared_memory(gnm, c3):
    reg, lpm, starts, sites, rec, keys = c3
    ctx = gnm.Context(window_slots=2, placement=gnm.PLACE_SMEM)
    ctx.load(reg)
    ctx.rmi_train(to_dev(keys), root_kind=gnm.ROOT_LINEAR, n_leaves=65536, leaf_iters=2)
    with pytest.raises(gnm.GnmError, match="too large for shared memory"):
        ctx.process(gnm.Records.to_device({k: v[:1000] for k, v in rec.items()}), 1)
    ctx.close()
