"""Shared test helpers: oracle results and comparison of the CUDA library's results
against them."""
import numpy as np

import oracle

RATE_RTOL = 1e-12  # rates: relative error bound of the FP64 rate against the FP64 oracle


def oracle_full(reg, rec, threshold=1e8, min_flows=1, lpm=None, n_threads=8, **kw):
    lpm = lpm or oracle.LPM(reg.prefix, reg.plen, reg.site)
    st, un = oracle.window(lpm, reg.local_prefix, reg.local_len, reg.n_sites, rec, n_threads=n_threads, **kw)
    r = oracle.rates(st)
    fl = oracle.flags(st, r, threshold, min_flows)
    return st, un, r, fl


def assert_rates_close(got, want, rtol=RATE_RTOL):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    gn, wn = np.isnan(got), np.isnan(want)
    np.testing.assert_array_equal(gn, wn)
    ok = ~wn
    diff = np.abs(got[ok] - want[ok])
    bound = rtol * np.abs(want[ok])
    assert np.all(diff <= bound), f"rate mismatch: max rel {np.max(diff / np.maximum(np.abs(want[ok]), 1e-300))}"


def assert_window_matches(dense, expect):
    st, un, r, f = dense
    ost, oun, orate, ofl = expect
    np.testing.assert_array_equal(st, ost)
    np.testing.assert_array_equal(un, oun)
    assert_rates_close(r, orate)
    np.testing.assert_array_equal(f, ofl)
