"""Pins for the oracle's relative KKT error (Section 5, "Criteria") on points
worked out by hand, term by term.

The market is already row-scaled (each row's largest utility is 1), so the
Section 5 preprocessing leaves it unchanged:

    buyer 0: goods {0, 1, 2}, u = (1, 1/2, 1/4), w_0 = 1
    buyer 1: goods {1, 2},    u = (1, 1/2),      w_1 = 2

With t_i = u_i^T x_i and y = w / t (the PDHCG setting of Section 5) the
t- and y-residuals vanish and

    r_primal = max_j |c_j - 1| / (1 + max(max_j c_j, 1)),          c = 1^T x
    r_dual   = max_j (p_j - M_j)_- / (1 + max(max_i y_i, max_j (p_j - M_j))),
               M_j = max_i u_ij y_i   (the last term is SIGNED in the paper)
    r_gap    = max_ij x_ij (p_j - u_ij y_i)_+
               / (1 + max(max_ij x_ij, max_ij (p_j - u_ij y_i)_+)).

Each point below is chosen so that a plausible slip changes a value:
  A  every c_j < 1, so dropping the |.| in the primal numerator gives a
     negative residual and dropping the 1 in its denominator changes it;
  B  a negative price makes |p_j - M_j| exceed max y, so an absolute value
     in the dual denominator (instead of the signed term) changes r_dual;
  C  max_j (p_j - M_j) < 0 and ||x||_inf dominates the gap denominator, so
     dropping ||x||_inf there changes r_gap; c_0 = 3 pins ||1^T x||_inf.
"""
import numpy as np
import pytest

from oracle import fisher as F

ROW_PTR = np.array([0, 3, 5], dtype=np.int64)
COL = np.array([0, 1, 2, 1, 2], dtype=np.int64)
VAL = np.array([1.0, 0.5, 0.25, 1.0, 0.5])
W = np.array([1.0, 2.0])


def _kkt(x, p):
    sc = F.preprocess(ROW_PTR, COL, VAL, W, 3)
    assert np.array_equal(sc.u, VAL)            # already row-scaled
    return F.kkt_error(sc, np.asarray(x, dtype=np.float64), np.asarray(p, dtype=np.float64))


def test_point_a_primal_below_one():
    # x = (1/2, 1/4, 1/2 | 1/2, 1/4)
    # t = (1/2 + 1/8 + 1/8, 1/2 + 1/8) = (3/4, 5/8);  y = (4/3, 16/5)
    # c = (1/2, 3/4, 3/4): r_primal = (1/2) / (1 + 1) = 1/4
    # u y = (4/3, 2/3, 1/3 | 16/5, 8/5);  M = (4/3, 16/5, 8/5)
    # p = (1, 3, 2): p - M = (-1/3, -1/5, 2/5); num = 1/3; den = 1 + max(16/5, 2/5) = 21/5
    #   r_dual = (1/3) / (21/5) = 5/63
    # (p_j - u y)_+ = (0, 7/3, 5/3 | 0, 2/5); x * that = (0, 7/12, 5/6 | 0, 1/10)
    #   r_gap = (5/6) / (1 + max(1/2, 7/3)) = (5/6) / (10/3) = 1/4
    k = _kkt([0.5, 0.25, 0.5, 0.5, 0.25], [1.0, 3.0, 2.0])
    assert k.r_primal == pytest.approx(0.25, rel=0, abs=1e-15)
    assert k.r_dual == pytest.approx(5.0 / 63.0, rel=0, abs=1e-15)
    assert k.r_gap == pytest.approx(0.25, rel=0, abs=1e-15)
    assert k.kkt == pytest.approx(0.25, rel=0, abs=1e-15)


def test_point_b_negative_price_signed_dual_denominator():
    # same x as A (t, y, c, M unchanged); p = (-4, 3, 2)
    # p - M = (-16/3, -1/5, 2/5): num = 16/3, signed max = 2/5
    #   r_dual = (16/3) / (1 + max(16/5, 2/5)) = (16/3) / (21/5) = 80/63
    #   (with |p - M| in the denominator it would be (16/3) / (19/3) = 16/19)
    # (p_j - u y)_+ = (0, 7/3, 5/3 | 0, 2/5): r_gap = 1/4 as in A
    k = _kkt([0.5, 0.25, 0.5, 0.5, 0.25], [-4.0, 3.0, 2.0])
    assert k.r_primal == pytest.approx(0.25, rel=0, abs=1e-15)
    assert k.r_dual == pytest.approx(80.0 / 63.0, rel=0, abs=1e-15)
    assert k.r_gap == pytest.approx(0.25, rel=0, abs=1e-15)
    assert k.kkt == pytest.approx(80.0 / 63.0, rel=0, abs=1e-15)


def test_point_c_negative_dual_term_and_x_norm():
    # x = (3, 1/4, 1/2 | 1/2, 1/4)
    # t = (3 + 1/8 + 1/8, 5/8) = (13/4, 5/8);  y = (4/13, 16/5)
    # c = (3, 3/4, 3/4): r_primal = 2 / (1 + max(3, 1)) = 1/2
    # u y = (4/13, 2/13, 1/13 | 16/5, 8/5);  M = (4/13, 16/5, 8/5)
    # p = (3/10, 1/5, 1/10): p - M = (-1/130, -3, -3/2), all negative
    #   num = 3; den = 1 + max(16/5, -1/130) = 21/5;  r_dual = 3 / (21/5) = 5/7
    # (p_j - u y)_+ = (0, 1/5 - 2/13, 1/10 - 1/13 | 0, 0) = (0, 3/65, 3/130 | 0, 0)
    # x * that = (0, 3/260, 3/260 | 0, 0);  max = 3/260
    #   r_gap = (3/260) / (1 + max(3, 3/65)) = (3/260) / 4 = 3/1040
    k = _kkt([3.0, 0.25, 0.5, 0.5, 0.25], [0.3, 0.2, 0.1])
    assert k.r_primal == pytest.approx(0.5, rel=0, abs=1e-15)
    assert k.r_dual == pytest.approx(5.0 / 7.0, rel=0, abs=1e-15)
    assert k.r_gap == pytest.approx(3.0 / 1040.0, rel=0, abs=1e-15)
    assert k.kkt == pytest.approx(5.0 / 7.0, rel=0, abs=1e-15)


def test_hand_equilibrium_has_zero_residuals():
    # Equilibrium of this market, found by hand.  Buyer 0 is the only buyer of
    # good 0, so if it bought nothing else p_0 = w_0 = 1.  Buyer 1 then buys
    # goods 1 and 2 with equal bang-per-buck, 1 / p_1 = (1/2) / p_2, and spends
    # w_1 = 2 = p_1 + p_2: p = (1, 4/3, 2/3).  Buyer 0's bang-per-buck is 1 on
    # good 0 against (1/2) / (4/3) = 3/8 and (1/4) / (2/3) = 3/8, so it indeed
    # buys good 0 only.  x = (1, 0, 0 | 1, 1):  t = (1, 3/2), y = (1, 4/3)
    # c = (1, 1, 1);  M = (1, 4/3, 2/3) = p;  every x_ij > 0 has p_j = u_ij y_i.
    k = _kkt([1.0, 0.0, 0.0, 1.0, 1.0], [1.0, 4.0 / 3.0, 2.0 / 3.0])
    assert k.r_primal == pytest.approx(0.0, abs=1e-15)
    assert k.r_dual == pytest.approx(0.0, abs=1e-15)
    assert k.r_gap == pytest.approx(0.0, abs=1e-15)


def test_clearing_allocation_at_wrong_prices():
    # x = (1, 0, 1 | 1, 0) clears every good: c = (1, 1, 1), r_primal = 0.
    # t = (1 + 1/4, 1) = (5/4, 1);  y = (4/5, 2)
    # u y = (4/5, 2/5, 1/5 | 2, 1);  M = (4/5, 2, 1)
    # p = (4/5, 2, 1/5): p - M = (0, 0, -4/5): buyer 1 would rather buy good 2
    #   r_dual = (4/5) / (1 + max(2, 0)) = 4/15
    # gap: x_ij > 0 only where p_j = u_ij y_i, so r_gap = 0
    k = _kkt([1.0, 0.0, 1.0, 1.0, 0.0], [0.8, 2.0, 0.2])
    assert k.r_primal == pytest.approx(0.0, abs=1e-15)
    assert k.r_gap == pytest.approx(0.0, abs=1e-15)
    assert k.r_dual == pytest.approx(4.0 / 15.0, rel=0, abs=1e-15)


def test_planted_denominator_slip_is_caught():
    """A copy of the dual residual with |p - M| in its denominator (a plausible
    misreading) fails point B's hand value: the pin above has teeth."""
    sc = F.preprocess(ROW_PTR, COL, VAL, W, 3)
    x = np.array([0.5, 0.25, 0.5, 0.5, 0.25])
    p = np.array([-4.0, 3.0, 2.0])
    t = F.row_dot(sc.row_ptr, sc.u, x)
    y = sc.w / t
    uy = sc.u * y[sc.rows]
    M = np.full(3, -np.inf)
    np.maximum.at(M, sc.col, uy)
    slipped = np.max(np.maximum(M - p, 0.0)) / (1.0 + max(np.max(y), np.max(np.abs(p - M))))
    assert abs(slipped - 80.0 / 63.0) > 0.1
    assert F.kkt_error(sc, x, p).r_dual == pytest.approx(80.0 / 63.0, abs=1e-15)
