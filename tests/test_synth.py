"""The seeded input generator: Philox4x32-10 known answers, determinism,
Assumption 1, and the shapes of the five workloads (scaled down)."""
import numpy as np

from paper_2506_06258_gb300 import synth as S


def test_philox_known_answers():
    """Known-answer vectors of Philox4x32-10 (Salmon et al., SC'11)."""
    assert S.philox4x32_10([0, 0, 0, 0], [0, 0]).tolist() == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert S.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2).tolist() == \
        [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert S.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0]).tolist() == \
        [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def _check_csr(mk):
    assert mk.row_ptr[0] == 0 and np.all(np.diff(mk.row_ptr) >= 1)        # no empty row
    assert np.all(np.bincount(mk.col, minlength=mk.m) >= 1)                # no empty column
    rows = np.repeat(np.arange(mk.n), np.diff(mk.row_ptr))
    same = rows[1:] == rows[:-1]
    assert np.all(np.diff(mk.col.astype(np.int64))[same] > 0)              # sorted, distinct
    assert np.all(mk.val > 0) and np.all(mk.w > 0)


def test_deterministic_and_valid():
    a, b = S.config1(), S.config1()
    assert np.array_equal(a.col, b.col) and np.array_equal(a.val, b.val) and np.array_equal(a.w, b.w)
    _check_csr(a)
    assert a.n == 200 and a.m == 100 and 0.15 < a.nnz / (200 * 100) < 0.25
    assert 0.5 <= a.w.min() and a.w.max() <= 1.5


def test_workload_shapes():
    c2 = S.config2(n=5000, m=300, d=100)
    _check_csr(c2)
    assert np.all(np.diff(c2.row_ptr) == 100)
    c3 = S.config3(n=20000, m=2000, nnz_target=2_000_000)
    _check_csr(c3)
    assert abs(c3.nnz - 2_000_000) <= 0.002 * 2_000_000
    d = np.diff(c3.row_ptr)
    assert d.min() >= 10 and d.max() <= 2000
    cd = np.bincount(c3.col, minlength=c3.m)
    assert cd.max() > 20 * np.median(cd)                                   # skewed popularity
    c4 = S.config4(n=500, d_other=10)
    _check_csr(c4)
    assert np.all(np.diff(c4.row_ptr) == 11)
    rows = np.repeat(np.arange(c4.n), 11)
    assert np.all(np.bincount(rows[c4.col == rows], minlength=c4.n) == 1)   # own good present
    assert np.all(c4.val >= 0.1) and np.all(c4.val <= 1.0) and np.all(c4.w == 1.0)
    bt = S.config5(B=6, n_range=(20, 80), m_range=(5, 30))
    for b in range(bt.B):
        _check_csr(bt.market(b))


def test_repair_assumption1():
    mk = S.Market(3, 3, np.array([0, 1, 1, 2]), np.array([0, 0], dtype=np.int32), np.array([0.5, 0.6]),
                  np.ones(3))
    fixed = S.repair_assumption1(mk, 1, S.LAW_UNIFORM, 0.0, 1.0)
    _check_csr(fixed)
