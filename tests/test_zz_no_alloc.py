"""The allocation-free entry point (gnm_window_process_noalloc) against the allocating
one (gnm_window_process), on two calls in a row.

It serves callers that cannot call cudaMalloc -- a process whose device memory belongs
to another allocator, or a latency-critical loop that cannot take cudaMalloc's implicit
device synchronisation: they pass every input and output themselves and the kernel keeps
its scratch in a fixed array inside the library. Results must equal the allocating
entry point's: integers bit-exact, rates within 1e-12 relative.
"""
import numpy as np
import pytest

import flowgen as fg
from helpers import assert_window_matches

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gnm():
    from paper_1108_1785_gb300 import build, gnm as g
    build.build()
    return g


def _dev_u32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def _noalloc(gnm, reg, starts_d, site_d, rec_dev):
    nk = 2 * reg.n_sites
    # the caller owns the outputs (here: torch allocations made before the call)
    stats = torch.full(((nk + 4) * 6,), -1, dtype=torch.int64, device="cuda")
    rate = torch.zeros(nk, dtype=torch.float64, device="cuda")
    flag = torch.full((nk,), 7, dtype=torch.uint8, device="cuda")
    gnm.window_process_noalloc(starts_d, site_d, reg.n_sites, reg.local_prefix, reg.local_len, rec_dev,
                               stats, rate, flag)
    torch.cuda.synchronize()
    st = stats.cpu().numpy().view(np.uint64).reshape(nk + 4, 6)
    return st[:nk].copy(), st[nk:, :3].copy(), rate.cpu().numpy(), flag.cpu().numpy()


@pytest.mark.parametrize("which", ["c1", "c2"])
def test_noalloc_equals_allocating_entry_point_on_two_calls(gnm, which):
    reg = fg.registry_c1() if which == "c1" else fg.registry_c2()
    starts, sites = gnm.registry_flatten(reg.prefix, reg.plen, reg.site, reg.n_sites)
    starts_d, site_d = _dev_u32(starts), _dev_u32(sites)
    ctx = gnm.Context(window_slots=4)
    ctx.load(reg)
    for call, seed in enumerate((41, 42)):  # two calls in a row share the fixed scratch
        rec = fg.make_records(reg, 150_000 + 3 * call, seed=seed, zipf_s=1.1 if which == "c1" else 1.0)
        d = gnm.Records.to_device(rec)
        got = _noalloc(gnm, reg, starts_d, site_d, d)
        ctx.process(d, call)
        assert_window_matches(got, ctx.dense(call))
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(gnm):
    reg = fg.registry_c1()
    starts, sites = gnm.registry_flatten(reg.prefix, reg.plen, reg.site, reg.n_sites)
    rec = gnm.Records.to_device(fg.window_records_c1(reg, n=1000))
    n_sites = 13102 + 1  # one site beyond GNM_NOALLOC_MAX_SITES
    stats = torch.empty(((2 * n_sites + 4) * 6,), dtype=torch.int64, device="cuda")
    rate = torch.empty(2 * n_sites, dtype=torch.float64, device="cuda")
    flag = torch.empty(2 * n_sites, dtype=torch.uint8, device="cuda")
    with pytest.raises(gnm.GnmError, match="allocation-free limit"):
        gnm.window_process_noalloc(_dev_u32(starts), _dev_u32(sites), n_sites, reg.local_prefix, reg.local_len, rec,
                                   stats, rate, flag)


def test_noalloc_site_ids_beyond_n_sites_count_as_unregistered(gnm):
    """The caller's registry arrays may hold site ids at or above the n_sites it passes:
    those ranges count as unregistered (unmatched classes 2 and 3), so no key reaches past
    the 2*n_sites + 4 rows of the scratch or of `stats`. The 2,000 prefixes of this registry
    do not overlap, so this equals the allocating entry point over the prefixes of the
    first 250 sites only."""
    import dataclasses
    reg = fg.registry_c1()
    starts, sites = gnm.registry_flatten(reg.prefix, reg.plen, reg.site, reg.n_sites)
    keep = reg.site < 250
    small = dataclasses.replace(reg, prefix=reg.prefix[keep], plen=reg.plen[keep], site=reg.site[keep], n_sites=250,
                                nested=reg.nested[keep])
    ctx = gnm.Context(window_slots=2)
    ctx.load(small)
    rec = fg.make_records(reg, 120_000, seed=43, zipf_s=1.1)
    d = gnm.Records.to_device(rec)
    got = _noalloc(gnm, small, _dev_u32(starts), _dev_u32(sites), d)
    ctx.process(d, 1)
    want = ctx.dense(1)
    assert_window_matches(got, want)
    assert int(want[1][2, 0] + want[1][3, 0]) > int(0.3 * rec["srcaddr"].size)  # many records left unmatched
    ctx.close()
