"""CPU-side checks of the C ABI library: it builds, loads, exports every entry point
declared in include/gnm.h, and its host-only registry step agrees with the oracle's
independent flattening (no GPU needed)."""
import ctypes as C
import ipaddress
import os
import re

import numpy as np
import pytest

import flowgen as fg
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gnm():
    from paper_1108_1785_gb300 import build, gnm as g
    build.build()
    return g


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "gnm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gnm_[a-z0-9_]+)\s*\(", txt)))


@pytest.mark.parametrize("name", ["libgnm.so", "libgnm_checked.so"])
def test_library_exports_every_declared_entry_point(gnm, name):
    """Both builds (the library and the one with device-side bounds checks) export every
    function gnm.h declares."""
    lib = C.CDLL(os.path.join(os.path.dirname(gnm.LIB_PATH), name))
    names = declared_functions()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared in gnm.h but not exported: {missing}"
    assert lib.gnm_checked_build() == (1 if "checked" in name else 0)


def test_config_defaults(gnm):
    c = gnm.Config()
    gnm.lib().gnm_config_default(C.byref(c))
    assert (c.min_avg_pkt_bytes, c.min_pkts, c.min_dur_ms, c.min_flows_to_flag) == (100, 10, 1000, 1)
    assert c.threshold_bps == 1e8 and c.window_slots == 64


@pytest.mark.parametrize("which", ["c1", "c2", "c3"])
def test_host_flatten_equals_oracle_flatten(gnm, which):
    reg = {"c1": fg.registry_c1, "c2": fg.registry_c2, "c3": fg.registry_c3}[which]()
    st, si = gnm.registry_flatten(reg.prefix, reg.plen, reg.site, reg.n_sites)
    ost, osi = oracle.LPM(reg.prefix, reg.plen, reg.site).flatten()
    np.testing.assert_array_equal(st, ost)
    np.testing.assert_array_equal(si, osi)


def test_host_flatten_nested_hand_case(gnm):
    ip = lambda s: int(ipaddress.IPv4Address(s))
    p = [ip("10.0.0.0"), ip("10.1.0.0"), ip("10.1.2.0"), ip("10.1.2.4"), ip("10.1.3.0"), ip("255.255.255.255"),
         ip("0.0.0.0")]
    l = [8, 16, 24, 30, 24, 32, 0]
    s = [0, 1, 2, 3, 4, 5, 6]
    st, si = gnm.registry_flatten(p, l, s, 7)
    want = [(0, 6), (ip("10.0.0.0"), 0), (ip("10.1.0.0"), 1), (ip("10.1.2.0"), 2), (ip("10.1.2.4"), 3),
            (ip("10.1.2.8"), 2), (ip("10.1.3.0"), 4), (ip("10.1.4.0"), 1), (ip("10.2.0.0"), 0),
            (ip("11.0.0.0"), 6), (ip("255.255.255.255"), 5)]
    assert list(zip(st.tolist(), si.tolist())) == want


@pytest.mark.parametrize("p,l,s,ns,msg", [
    ([0x0A000001], [24], [0], 1, "host bits"),
    ([0x0A000000], [33], [0], 1, "length"),
    ([0x0A000000] * 2, [8, 8], [0, 1], 2, "duplicate"),
    ([0x0A000000], [8], [3], 1, "site id"),
])
def test_host_flatten_rejects(gnm, p, l, s, ns, msg):
    with pytest.raises(gnm.GnmError, match=msg):
        gnm.registry_flatten(p, l, s, ns)


def test_empty_registry_is_one_gap(gnm):
    st, si = gnm.registry_flatten([], [], [], 1)
    assert st.tolist() == [0] and si.tolist() == [gnm.NO_SITE]


def test_create_without_gpu_fails_cleanly(gnm):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(gnm.GnmError, match="CUDA"):
        gnm.Context()
