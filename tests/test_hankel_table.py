"""The polynomial tables of H_0 and H_1 that the device special functions use
below x = 8 (paper_1602_05301_gb300/csrc/hankel_table.h): the committed header
is what its generator writes, and its pieces, evaluated in float64 the way the
device does (row from the bit fields of x, Horner's rule in t or u, the
logarithmic terms of the ascending series added below x = 2^-9), match H_0 and
H_1 from mpmath relative to |H_0|, |H_1|: 1e-15 for the FP64 tables, 3e-13 for
the mixed-precision ones, in every octave and at the interval ends."""
import os
import re
import struct
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1602_05301_gb300", "csrc")
HEADER = os.path.join(CSRC, "hankel_table.h")


def parse(name):
    text = open(HEADER).read()
    rows = int(re.search(r"kHankRows = (\d+)", text).group(1))
    emin = int(re.search(r"kHankMinExp = (-?\d+)", text).group(1))
    deg = int(re.search(r"kHankDeg%s = (\d+)" % name, text).group(1))
    body = re.search(r"kHankTab%s\[\d+\] = \{(.*?)\n\};" % name, text, re.S).group(1)
    vals = [float(v) for v in re.findall(r"[-+]?[0-9][-+0-9.e]*", body)]
    tab = np.array(vals).reshape(deg + 1, 2, rows, 2)   # [d][pair][row][component]
    return rows, emin, deg, tab


def evaluate(name, x):
    """H_0, H_1 from the table as the device forms them (one lane at a time)."""
    rows, emin, deg, tab = parse(name)
    gamma, two_pi = 0.57721566490153286061, 0.63661977236758134308
    out = np.zeros((x.size, 2), complex)
    for i, xi in enumerate(x):
        if xi < 2.0 ** emin:
            v, row = -0.25 * xi * xi, rows - 1
        else:
            hi = struct.unpack(">II", struct.pack(">d", xi))[0]
            row = ((hi >> 17) & 0x3FFF) - ((1023 + emin) << 3)
            E = ((hi >> 20) & 0x7FF) - 1023
            v = xi * (16.0 / 2 ** E) - (17 + 2 * (row & 7))
        c = tab[deg, :, row, :].copy()
        for d in range(deg - 1, -1, -1):
            c = c * v + tab[d, :, row, :]
        if xi < 2.0 ** emin:
            j0s, r0s, p1s, r1s = c[0, 0], c[0, 1], c[1, 0], c[1, 1]
            lx = np.log(0.5 * xi)
            J1 = 0.5 * xi * p1s
            h0 = j0s + 1j * two_pi * ((lx + gamma) * j0s - r0s)
            h1 = J1 + 1j * (-two_pi / xi + two_pi * lx * J1 - 0.5 * xi * 0.5 * two_pi * r1s)
        else:
            h0, h1 = c[0, 0] + 1j * c[0, 1], c[1, 0] + 1j * c[1, 1]
        out[i] = h0, h1
    return out


@pytest.mark.parametrize("name,bound", [("64", 1e-15), ("Mx", 3e-13)])
def test_table_matches_mpmath(name, bound):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    rng = np.random.default_rng(11)
    ends = [2.0 ** E * (1 + j / 8) for E in range(-9, 3) for j in range(8)]
    x = np.concatenate([np.geomspace(1e-7, 8.0, 1500, endpoint=False),
                        rng.uniform(0.0, 8.0, 300), np.linspace(2.0, 8.0, 300, endpoint=False),
                        ends, [np.nextafter(e, 0) for e in ends], [8.0 - 1e-12]])
    x = x[(x > 0) & (x < 8)]
    h = evaluate(name, x)
    ref = np.array([[complex(mp.hankel1(0, xi)), complex(mp.hankel1(1, xi))] for xi in x])
    err = np.abs(h - ref) / np.abs(ref)
    print("%s: max relative error %.2e (x < 2^-9: %.2e)" % (name, err.max(), err[x < 2.0 ** -9].max()))
    assert err.max() < bound


def test_header_is_the_generator_output():
    pytest.importorskip("mpmath")
    r = subprocess.run([sys.executable, os.path.join(CSRC, "gen_hankel_table.py")],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    assert r.stdout == open(HEADER).read()
