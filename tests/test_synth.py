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


def test_jd_activity_profile_matches_the_table():
    """Every prefix of the n most active users holds the table's pair count
    (Section 5.2, Table tab:fisher); every user clicked something."""
    d = S.jd_activity_profile()
    assert len(d) == S.JD_USERS[-1] and d.min() >= 1
    assert [int(d[:n].sum()) for n in S.JD_USERS] == list(S.JD_NNZ)
    assert d[0] > 50 * np.median(d)                                        # heavy-tailed activity


def test_jd_like_market_prefixes():
    small = S.jd_like_market(2000)
    _check_csr(small)
    assert small.n == 2000 and small.nnz == S.JD_NNZ[0]
    assert abs(small.m / S.JD_GOODS[0] - 1.0) <= 0.15
    assert np.all(small.val == np.floor(small.val)) and small.val.min() >= 1.0      # click counts
    assert small.w.max() < 1.0
    again = S.jd_like_market(2000)
    assert np.array_equal(small.col, again.col) and np.array_equal(small.val, again.val)
    mid = S.jd_like_market(20000)
    assert mid.nnz == S.JD_NNZ[2] and abs(mid.m / S.JD_GOODS[2] - 1.0) <= 0.15
    # rows are not in activity order, but sorting them back recovers the profile
    rank = mid.meta["activity_rank"]
    deg = np.diff(mid.row_ptr)
    assert not np.all(np.diff(deg) <= 0)
    assert np.array_equal(np.sort(deg)[::-1], np.sort(S.jd_activity_profile()[:20000])[::-1])
    assert np.array_equal(deg[np.argsort(rank)], S.jd_activity_profile()[:20000])


def test_jd_like_market_full_log_has_every_product():
    full = S.jd_like_market()
    _check_csr(full)
    assert full.n == S.JD_USERS[-1] and full.m == S.JD_GOODS[-1]
    assert 0 <= full.nnz - S.JD_NNZ[-1] <= 0.001 * S.JD_NNZ[-1]             # one-click repairs only


def test_ad_random_instance():
    mk, (erp, ecol, ev) = S.ad_random_instance(300, 120, 0.2, 0.5, seed=3)
    _check_csr(mk)
    assert np.all(np.diff(erp) >= 1) and np.all(np.bincount(ecol, minlength=120) >= 1)
    assert np.allclose(np.bincount(ecol, weights=ev, minlength=120), 1.0, atol=1e-12)   # unit supply per good
    rows = np.repeat(np.arange(300), np.diff(erp))
    assert np.allclose(mk.w, np.bincount(rows, weights=ev, minlength=300)) and np.isclose(mk.w.sum(), 120)
    assert 0.4 < len(ecol) / (300 * 120) < 0.6 and 0.15 < mk.nnz / (300 * 120) < 0.25
