"""Writes hankel_table.h: the polynomial pieces of H_0 = J_0 + i Y_0 and
H_1 = J_1 + i Y_1 (DLMF 10.4.3) that the device special functions evaluate
below x = 8.

* 2^-9 <= x < 8: eight intervals per octave, [2^E (1 + j/8), 2^E (1 + (j+1)/8))
  for E = -9..2 (the interval index is a bit field of x: its exponent and top
  three mantissa bits). On each, J_0, Y_0, J_1, Y_1 are truncated Chebyshev
  series of degree D in t = (x - centre) / half-width, written out as
  monomials in t. The partition is geometric, so the logarithmic singularity
  of Y at 0 lies 17 half-widths from every interval's centre and one degree
  serves all octaves.
* x < 2^-9: the ascending series (DLMF 10.2.2, 10.8.1) in u = -x^2/4 of the
  four entire functions J_0, J_1 / (x/2), R_0 = sum H_k u^k / (k!)^2 and
  R_1 = sum (psi(k+1) + psi(k+2)) u^k / (k! (k+1)!), each a truncated
  Chebyshev series of degree D on u in [-1, 0] written out as monomials in u
  (the logarithmic terms are added by the caller).

Two tables: degree 10 (truncation near 1e-16 of |H_0|, |H_1|) for the FP64
path and degree 8 (near 1e-13) for the mixed-precision path, whose Hankel
values are rounded to FP32 after an FP64 recurrence. Values come from mpmath
at 40 digits. Run: python gen_hankel_table.py > hankel_table.h
"""
import mpmath as mp

mp.mp.dps = 40
NCHEB = 40          # Chebyshev coefficients computed before truncation
PER_OCTAVE = 8
OCTAVES = tuple(range(-9, 3))   # [2^-9, 2^-8), ..., [4, 8)
DEGREES = {"64": 10, "Mx": 8}


def chebyshev_coefficients(f, a, b, n=NCHEB):
    """c_j of f(mid + half t) ~ sum c_j T_j(t) on [a, b] (interpolation at n
    Chebyshev points, which for smooth f matches the series to rounding)."""
    mid, half = (a + b) / 2, (b - a) / 2
    th = [mp.pi * (k + mp.mpf(1) / 2) / n for k in range(n)]
    fv = [f(mid + half * mp.cos(t)) for t in th]
    return [(2 if j else 1) * mp.fsum(fv[k] * mp.cos(j * th[k]) for k in range(n)) / n
            for j in range(n)]


def to_monomial(c, deg, shift=None):
    """sum_{j<=deg} c_j T_j(s) as monomial coefficients in s, or, with
    shift=(p, q), in w where s = p w + q."""
    T = [[mp.mpf(1)], [mp.mpf(0), mp.mpf(1)]]
    while len(T) <= deg:
        a, b = T[-1], T[-2]
        t = [mp.mpf(0)] * (len(a) + 1)
        for i, v in enumerate(a):
            t[i + 1] += 2 * v
        for i, v in enumerate(b):
            t[i] -= v
        T.append(t)
    m = [mp.mpf(0)] * (deg + 1)
    for j in range(deg + 1):
        for i, v in enumerate(T[j]):
            m[i] += c[j] * v
    if shift is None:
        return m
    p, q = shift
    out = [mp.mpf(0)] * (deg + 1)
    for i, v in enumerate(m):   # (p w + q)^i by the binomial theorem
        for r in range(i + 1):
            out[r] += v * mp.binomial(i, r) * p ** r * q ** (i - r)
    return out


def series_functions():
    """The four entire functions of u of the ascending series."""
    def make(kind):
        def f(u):
            s, h = mp.mpf(0), mp.mpf(0)
            psi = -mp.euler
            psis = [psi]
            for k in range(1, 60):
                psis.append(psis[-1] + mp.mpf(1) / k)   # psi(k+1)
            for k in range(50):
                if k:
                    h += mp.mpf(1) / k
                f0 = 1 / mp.factorial(k) ** 2
                f1 = 1 / (mp.factorial(k) * mp.factorial(k + 1))
                c = {"J0": f0, "P1": f1, "R0": h * f0, "R1": (psis[k] + psis[k + 1]) * f1}[kind]
                s += c * u ** k
            return s
        return f
    return [make(k) for k in ("J0", "R0", "P1", "R1")]


def intervals():
    for E in OCTAVES:
        for j in range(PER_OCTAVE):
            a = mp.mpf(2) ** E * (1 + mp.mpf(j) / PER_OCTAVE)
            yield a, a + mp.mpf(2) ** E / PER_OCTAVE


def rows(deg):
    """Per row, the four polynomials (J0, Y0, J1, Y1 or the series four)."""
    out = []
    fs = [lambda x: mp.besselj(0, x), lambda x: mp.bessely(0, x),
          lambda x: mp.besselj(1, x), lambda x: mp.bessely(1, x)]
    for a, b in intervals():
        out.append([to_monomial(chebyshev_coefficients(f, a, b), deg) for f in fs])
    # series row: u in [-1, 0], s = 2 u + 1
    out.append([to_monomial(chebyshev_coefficients(f, mp.mpf(-1), mp.mpf(0)), deg,
                            shift=(mp.mpf(2), mp.mpf(1))) for f in series_functions()])
    return out


def emit():
    nrow = len(list(intervals())) + 1
    lines = [
        "// Generated by gen_hankel_table.py (mpmath, 40 digits); do not edit.",
        "// Polynomial pieces of H_0 and H_1 below x = 8: rows 0..%d are the" % (nrow - 2),
        "// intervals [2^E (1 + j/8), 2^E (1 + (j+1)/8)), E = %d..%d (row 8 (E + %d) + j)," % (
            OCTAVES[0], OCTAVES[-1], -OCTAVES[0]),
        "// in t = 16 x / 2^E - 17 - 2 j; row %d is the economised ascending series in" % (nrow - 1),
        "// u = -x^2/4 (x < 2^%d). Entry [(d * 2 + q) * kHankRows + row] holds the" % OCTAVES[0],
        "// degree-d coefficients of pair q: (J0, Y0), (J1, Y1) on intervals; (J0, R0),",
        "// (J1 / (x/2), R1) on the series row.",
        "#pragma once",
        "constexpr int kHankRows = %d, kHankSeriesRow = %d, kHankMinExp = %d;" % (
            nrow, nrow - 1, OCTAVES[0]),
    ]
    for name, deg in DEGREES.items():
        R = rows(deg)
        lines.append("constexpr int kHankDeg%s = %d;" % (name, deg))
        lines.append("static __device__ const double2 kHankTab%s[%d] = {" % (name, (deg + 1) * 2 * nrow))
        for d in range(deg + 1):
            for q in range(2):
                vals = []
                for r in R:
                    vals.append("{%s, %s}" % (mp.nstr(r[2 * q][d], 17, min_fixed=1, max_fixed=0),
                                              mp.nstr(r[2 * q + 1][d], 17, min_fixed=1, max_fixed=0)))
                lines.append("    " + ", ".join(vals) + ",")
        lines.append("};")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    print(emit(), end="")
