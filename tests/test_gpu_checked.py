"""The build with device-side bounds checks (libgnm_checked.so, GNM_CHECKED=1).

Its kernels test every index where they trust data and, on a failure, skip the access and
record it; readouts then return GNM_E_INTERNAL. Run in child processes (the binding loads
one library per process):
- the parity cases of the C1, C2 and C3 registries under the checked build: no check fails
  and every result still equals the oracle;
- a corrupt learned-index routing word planted from the host: the check catches the model
  number beyond the model arrays, the lookups fall back to the full search, and the window
  still equals the oracle -- with no access out of bounds;
- the default build refuses to plant it.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import flowgen as fg
from helpers import assert_window_matches, oracle_full

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CHECKED = os.environ.get("GNM_CHECKED") == "1"


@pytest.fixture(scope="module")
def gnm():
    from paper_1108_1785_gb300 import build, gnm as g
    build.build()
    return g


def _child(args, timeout=1500):
    env = dict(os.environ, GNM_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"] + args,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    print("\nchecked build:", r.stdout.strip().splitlines()[-1])
    return r.stdout


@pytest.mark.skipif(CHECKED, reason="runs the checked build in a child process")
def test_checked_build_parity_cases(gnm):
    out = _child([
        "tests/test_gpu_checked.py::test_in_checked_build",
        "tests/test_gpu_window.py::test_hand_window",
        "tests/test_gpu_window.py::test_c1_window_all_variants",
        "tests/test_gpu_window.py::test_c1_ragged_and_unaligned",
        "tests/test_gpu_window.py::test_c2_hour_batched_bitexact",
        "tests/test_gpu_window.py::test_lookup_matches_oracle",
        "tests/test_gpu_window.py::test_one_slot_reused_after_global_sums",
        "tests/test_gpu_window.py::test_hash24_lookup_windows_match_oracle",
        "tests/test_gpu_rmi.py::test_rmi_window_equals_bsearch_and_oracle",
        "tests/test_gpu_rmi.py::test_rmi_window_fallback_exact",
        "tests/test_gpu_rmi.py::test_large_key_space_windows",
        "tests/test_gpu_rmi.py::test_mlp_root_window_exact",
        "tests/test_gpu_rate_stats.py::test_sparse_rate_stats_match_oracle",
        "tests/test_gpu_stream.py",
        "tests/test_zz_no_alloc.py",
    ])
    import re
    m = re.search(r"(\d+) passed", out)
    assert m and int(m.group(1)) >= 300 and "failed" not in out, out[-2000:]


@pytest.mark.skipif(CHECKED, reason="runs the checked build in a child process")
def test_checked_build_catches_a_corrupt_model_number(gnm):
    _child(["tests/test_gpu_checked.py::test_corrupt_split_base_is_caught"], timeout=900)


@pytest.mark.skipif(CHECKED, reason="the default build only")
def test_default_build_refuses_corruption(gnm):
    assert not gnm.checked_build()
    reg = fg.registry_c1()
    ctx = gnm.Context(window_slots=1)
    ctx.load(reg)
    with pytest.raises(gnm.GnmError, match="checked build"):
        ctx.debug_corrupt(gnm.DEBUG_RMI_SPLIT_BASE, 0, 0x7FFFFFF0)
    assert ctx.device_checks() == 0
    ctx.close()


# ------------------------------------------------ run in the child (GNM_CHECKED=1)

@pytest.mark.skipif(not CHECKED, reason="runs in the checked build's child process")
def test_in_checked_build(gnm):
    assert gnm.checked_build()


@pytest.mark.skipif(not CHECKED, reason="runs in the checked build's child process")
def test_corrupt_split_base_is_caught(gnm):
    """The routing word of the busiest split leaf of the learned index now names a model
    far beyond the model arrays. Every lookup through it trips the model-number check: the
    lookup takes the full search instead, the readout reports the check once, and the
    window's results equal the oracle's."""
    assert gnm.checked_build()
    reg = fg.registry_c3()
    rec = fg.make_records(reg, 1_000_000, seed=31, p_reg=0.9, zipf_s=0.9)
    ctx = gnm.Context(window_slots=2)
    ctx.load(reg)
    keys = fg.lookup_keys_c3(reg, 2_000_000)
    ctx.rmi_train(torch.from_numpy(keys.view(np.int32)).cuda(), n_leaves=4096)
    m = ctx.rmi_export()
    split = np.nonzero(m["split"])[0]
    assert split.size > 0
    root = m["root"]
    from oracle import rmi_ref
    leaf = rmi_ref.root_linear(float(root[0]), float(root[1]), keys, 4096)
    busiest = split[np.argmax(np.bincount(leaf, minlength=4096)[split])]
    assert ctx.device_checks() == 0
    ctx.debug_corrupt(gnm.DEBUG_RMI_SPLIT_BASE, int(busiest), 0x7FFFFFF0)
    ctx.process(gnm.Records.to_device(rec), 1)
    with pytest.raises(gnm.GnmError, match="learned-index model number beyond the models"):
        ctx.device_checks()
    assert ctx.device_checks() == 0  # the word was cleared by the report
    assert_window_matches(ctx.dense(1), oracle_full(reg, rec))
    ctx.close()
