"""Oracle: counts at any size by exact interpolation (test infrastructure only).

Section "Gathering Kernel Statistics": every count is a piecewise
quasi-polynomial in the size parameters.  On one residue class
n = r + P*k (P the period) and away from the small-size pieces it is an
ordinary polynomial of some degree d in n, so d + 1 brute-force samples fix it
exactly; one more sample checks the degree.  Interpolation is Lagrange's in
exact rationals.
"""
from fractions import Fraction


def lagrange_eval(xs, ys, x):
    x = Fraction(x)
    total = Fraction(0)
    for i, (xi, yi) in enumerate(zip(xs, ys)):
        term = Fraction(yi)
        for j, xj in enumerate(xs):
            if j != i:
                term *= (x - xj) / Fraction(xi - xj)
        total += term
    return total


def extrapolate(fn, target, period, degree, start):
    """Exact value of the quasi-polynomial fn at `target`, from brute-force
    samples fn(n) at n = start + period*k (k = 0..degree+1), all in the
    residue class of target modulo period.  Raises if the extra sample does
    not lie on the degree-`degree` interpolant."""
    if (target - start) % period:
        raise ValueError("start and target are in different residue classes")
    xs = [start + period * k for k in range(degree + 2)]
    ys = [fn(x) for x in xs]
    check = lagrange_eval(xs[:-1], ys[:-1], xs[-1])
    if check != ys[-1]:
        raise ValueError("samples are not a degree-%d polynomial on this class" % degree)
    v = lagrange_eval(xs, ys, target)
    if v.denominator != 1:
        raise ValueError("non-integer extrapolated count")
    return int(v)
