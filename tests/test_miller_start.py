"""The start index of Miller's backward recurrence (miller_start in
paper_1602_05301_gb300/csrc/special.cuh), restated here: with m = max(pmax, x),
N = m + ceil(20 / arccosh(m / x)) + 2 where x <= m / 2 (Debye's asymptotics,
DLMF 10.19.3: above the turning point each order n shrinks J_n and grows Y_n by
e^{arccosh(n / x)}), else m + 12 + 2 sqrt(40 x), rounded up to even. Checked
against J_m from mpmath at 40 digits: the recurrence started at N, normalised
by the Neumann sum (DLMF 10.12.4), gives every J_m, m <= pmax, to a relative
2e-16, and a start two orders lower already does."""
import math

import numpy as np
import pytest


def start(pmax, x):
    m = max(pmax, int(x))
    if 2.0 * x <= m:
        n = m + 2 + int(math.ceil(20.0 / math.acosh(m / x)))
    else:
        n = m + 12 + int(2.0 * math.sqrt(40.0 * x))
    return n + (n & 1)


def miller(mp, x, M, N):
    x = mp.mpf(x)
    fn1, fn, s = mp.mpf(0), mp.mpf(10) ** -30, mp.mpf(0)
    row = {}
    for n in range(N, 0, -1):
        fm = 2 * n / x * fn - fn1
        if n % 2 == 0:
            s += fn
        if n - 1 <= M:
            row[n - 1] = fm
        fn1, fn = fn, fm
    norm = fn + 2 * s
    return [row[m] / norm for m in range(M + 1)]


@pytest.mark.parametrize("pmax", [1, 3, 8, 16, 42, 100])
def test_start_index_reaches_full_precision(pmax):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for x in np.geomspace(1e-6, 0.5 * pmax, 5):
        jex = [mp.besselj(m, x) for m in range(pmax + 1)]
        N = start(pmax, float(x))
        err = max(abs(a - b) / abs(b) for a, b in zip(miller(mp, x, pmax, N), jex))
        assert err < 2e-16, (pmax, x, N, float(err))
        # the start keeps a margin: two orders fewer are still enough
        err2 = max(abs(a - b) / abs(b) for a, b in zip(miller(mp, x, pmax, N - 2), jex))
        assert err2 < 2e-16, (pmax, x, N - 2, float(err2))
