"""The rate step alone (gnm_rates) against the oracle's FP64 expression, bit for bit.

The library forms (RN(e_octets) * 8000) / RN(e_dur_ms) on the integer units: the two
conversions, the product and the division each rounded to nearest as binary64 does
(Sec. III.B.1 and Sec. III.B.2.1: transfer rate = bits over seconds; one rounding per
operation is the reading of the rate's arithmetic). The oracle computes the same
expression with the host's IEEE 754 double arithmetic, so every bit must agree: random sums
of every magnitude, sums whose conversion rounds (above 2^53), quotients near the ends of a
binade, and the special cases (no eligible duration: NaN; no eligible octets: +0)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gnm():
    from paper_1108_1785_gb300 import build, gnm as g
    build.build()
    return g


def _gpu_rates(gnm, eo, ed):
    t_eo = torch.from_numpy(eo.view(np.int64)).cuda()
    t_ed = torch.from_numpy(ed.view(np.int64)).cuda()
    out = torch.empty(eo.size, dtype=torch.float64, device="cuda")
    gnm.rates(t_eo, t_ed, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _oracle_rates(eo, ed):
    st = np.zeros((eo.size, 6), np.uint64)
    st[:, 4] = eo
    st[:, 5] = ed
    return oracle.rates(st)


def _assert_bits_equal(got, want):
    gb, wb = got.view(np.uint64), want.view(np.uint64)
    bad = np.nonzero(gb != wb)[0]
    assert bad.size == 0, f"{bad.size} rates differ, first at {bad[0]}: {got[bad[0]]!r} != {want[bad[0]]!r}"


def _random_width(rng, n, lo, hi):
    """u64 values whose bit length is uniform in [lo, hi] (0 gives the value 0)."""
    w = rng.integers(lo, hi + 1, n)
    v = rng.integers(0, 2**63, n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, n, dtype=np.uint64)
    top = np.where(w > 0, np.uint64(1) << np.maximum(w - 1, 0).astype(np.uint64), np.uint64(0))
    low = np.where(w > 1, v & (top - np.uint64(1)), np.uint64(0))
    return (top | low).astype(np.uint64)


def test_rates_random_magnitudes_bit_exact(gnm):
    rng = np.random.default_rng(2024)
    n = 4_000_000
    eo = _random_width(rng, n, 0, 64)
    ed = _random_width(rng, n, 1, 64)
    _assert_bits_equal(_gpu_rates(gnm, eo, ed), _oracle_rates(eo, ed))


def test_rates_window_sized_sums_bit_exact(gnm):
    """Sums of the shape windows produce: up to 2^32 flows of octets below 2^32 and
    durations below 2^32 ms."""
    rng = np.random.default_rng(7)
    n = 2_000_000
    flows = rng.integers(1, 1 << 22, n).astype(np.uint64)
    eo = (flows * rng.integers(1, 1 << 32, n).astype(np.uint64)) >> rng.integers(0, 20, n).astype(np.uint64)
    ed = (flows * rng.integers(1000, 60001, n).astype(np.uint64))
    _assert_bits_equal(_gpu_rates(gnm, eo, ed), _oracle_rates(eo, ed))


def test_rates_special_and_boundary_operands(gnm):
    vals = [0, 1, 2, 3, 5, 7, 125, 8000, (1 << 32) - 1, 1 << 32, (1 << 52) - 1, 1 << 52, (1 << 52) + 1,
            (1 << 53) - 1, 1 << 53, (1 << 53) + 1, (1 << 53) + 3, (1 << 54) - 1, (1 << 63) - 1, 1 << 63,
            (1 << 64) - 1, (1 << 64) - 2, 0xAAAAAAAAAAAAAAAA, 0x5555555555555555, 0x0010000000000001]
    eo = np.array([a for a in vals for _ in vals], np.uint64)
    ed = np.array([b for _ in vals for b in vals], np.uint64)
    # quotients with an all-ones or all-zeros significand tail: b = a * 8000 +- small
    rng = np.random.default_rng(3)
    a = rng.integers(1, 1 << 50, 20000).astype(np.uint64)
    eo = np.concatenate([eo, a, a, a])
    ed = np.concatenate([ed, a * np.uint64(8000) + np.uint64(1), a * np.uint64(8000) - np.uint64(1),
                         a * np.uint64(4000) + np.uint64(1)])
    got, want = _gpu_rates(gnm, eo, ed), _oracle_rates(eo, ed)
    _assert_bits_equal(got, want)
    assert np.all(np.isnan(got[ed == 0])) and np.all(got[(eo == 0) & (ed != 0)].view(np.uint64) == 0)


def test_rates_rejects_bad_arguments(gnm):
    t = torch.zeros(4, dtype=torch.int64, device="cuda")
    r = torch.zeros(4, dtype=torch.float64, device="cuda")
    lib = gnm.lib()
    assert lib.gnm_rates(None, None, 0, None, None) == 0                      # nothing to do
    assert lib.gnm_rates(None, t.data_ptr(), 4, r.data_ptr(), None) == 1      # NULL array
    assert lib.gnm_rates(t.data_ptr() + 4, t.data_ptr(), 2, r.data_ptr(), None) == 1  # misaligned
