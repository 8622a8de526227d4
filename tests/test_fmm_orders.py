"""Level-dependent box orders (Sec. 7.1, "Maintaining Expansion Accuracy"),
computed by the library on the host, checked against the truncation bound
evaluated independently with mpmath at 50 digits:
  B_n(R) = |H_n(3 k R)| * max_{y <= sqrt2 k R} |J_n(y)|,
eps = max_{n > p_fmm} B_n at k R = min(k R_finest, 1); each level's order p
(box order minus p_add) must satisfy B_n <= eps for n > p and B_p > eps
(minimality)."""
import math

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 50


def log_bound(n, kR):
    a, b = 3 * kR, math.sqrt(2.0) * kR
    lh = mpmath.log(abs(mpmath.hankel1(n, a)))
    # beyond n = b, J_n increases on [0, b]; below it the bound 1 is used
    lj = mpmath.log(abs(mpmath.besselj(n, b))) if n > b else 0
    return float(lh + lj)


@pytest.fixture(scope="module")
def qbxmod():
    from paper_1602_05301_gb300 import qbx
    try:
        qbx.library()
    except RuntimeError as e:
        pytest.skip(str(e))
    return qbx


CASES = [
    # k, root side, levels, p_fmm, p_add: starfish k=10, k=50, 200 ellipses k=20, a k=40 curve
    (10.0, 4.0, 8, 20, 30),
    (50.0, 4.0, 10, 30, 40),
    (20.0, 102.0, 13, 30, 40),
    (40.0, 2.3, 9, 20, 30),
]


@pytest.mark.parametrize("k,side,nl,p_fmm,p_add", CASES)
def test_orders_meet_the_truncation_bound(qbxmod, k, side, nl, p_fmm, p_add):
    pb = qbxmod.qbx_fmm_level_orders(k, side, nl, p_fmm, p_add)
    assert pb[0] == 0 and pb[1] == 0
    assert 0.5 * k * side / 2 ** (nl - 1) <= 1.0
    assert pb[nl - 1] == p_fmm + p_add           # finest level below k R = 1 keeps p_fmm
    assert np.all(np.diff(pb[2:]) <= 0)           # coarser boxes never get lower orders
    kR = lambda l: 0.5 * k * side / 2 ** l
    leps = max(log_bound(n, kR(nl - 1)) for n in range(p_fmm + 1, p_fmm + 6))
    for l in range(2, nl - 1):
        p = int(pb[l]) - p_add
        r = kR(l)
        above = [log_bound(n, r) for n in range(p + 1, p + 9)]
        assert max(above) <= leps + 1e-9, (l, p, max(above), leps)
        if p > p_fmm:
            assert log_bound(p, r) > leps, (l, p)


def test_low_frequency_limit_keeps_p_fmm(qbxmod):
    # boxes far below a wavelength everywhere: every level gets p_fmm (+1 at most,
    # from the O((kR)^2) growth of the bound with kR)
    pb = qbxmod.qbx_fmm_level_orders(1e-3, 1.0, 10, 20, 30)
    assert np.all(pb[2:] >= 50) and np.all(pb[2:] <= 51)


def test_high_frequency_finest_level_gets_the_bound_order(qbxmod):
    # finest boxes at k R = 4: eps comes from k R = 1, the finest level needs more than p_fmm
    k, side, nl, p_fmm, p_add = 8.0, 16.0, 5, 20, 30
    pb = qbxmod.qbx_fmm_level_orders(k, side, nl, p_fmm, p_add)
    leps = max(log_bound(n, 1.0) for n in range(p_fmm + 1, p_fmm + 6))
    r = 0.5 * k * side / 2 ** (nl - 1)
    p = int(pb[nl - 1]) - p_add
    assert p > p_fmm
    assert max(log_bound(n, r) for n in range(p + 1, p + 9)) <= leps + 1e-9
    assert log_bound(p, r) > leps


def test_rejects_boxes_beyond_the_largest_order(qbxmod):
    with pytest.raises(qbxmod.QBXError):
        qbxmod.qbx_fmm_level_orders(100.0, 1000.0, 6, 30, 40)
    with pytest.raises(qbxmod.QBXError):
        qbxmod.qbx_fmm_level_orders(0.0, 1.0, 6, 30, 40)
