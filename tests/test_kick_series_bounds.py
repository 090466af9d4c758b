"""The kick's short Taylor polynomials (CPU, 50-digit mpmath): each is used
only where its truncation error is below a quarter of the unit roundoff of
the factor it forms; larger arguments go to the library's sincos / expm1.

For each (precision, function, degree, range) the line-solve kernels use,
the textbook Taylor polynomial of that degree is compared with the function
over the whole range, and the largest error must stay below the stated
bound; at four times the range it must not (so the range test in front of
each polynomial is needed, and the check is not vacuous).  The FP64 cosine
keeps one term more than the bound needs (through x^8 already meets it).
The kernels' own evaluation of these polynomials is checked against the
oracle by the GPU parity tests, including phases far outside the ranges
(g = 3000)."""
import pytest

mp = pytest.importorskip("mpmath")
mp.mp.dps = 50

U32, U64 = mp.mpf(2) ** -24, mp.mpf(2) ** -53  # unit roundoffs (half the spacing of numbers at 1)


def taylor(kind, x, degree):
    x = mp.mpf(x)
    s = mp.mpf(0)
    for k in range(degree + 1):
        if kind == "sin" and k % 2 == 1:
            s += (-1) ** (k // 2) * x ** k / mp.factorial(k)
        elif kind == "cos" and k % 2 == 0:
            s += (-1) ** (k // 2) * x ** k / mp.factorial(k)
        elif kind == "expm1m" and k >= 1:  # exp(-x) - 1
            s += (-x) ** k / mp.factorial(k)
    return s


def exact(kind, x):
    x = mp.mpf(x)
    return {"sin": mp.sin, "cos": mp.cos, "expm1m": lambda t: mp.expm1(-t)}[kind](x)


def worst_error(kind, degree, rng, relative_to):
    worst = mp.mpf(0)
    for i in range(-200, 201):
        x = rng * mp.mpf(i) / 200
        if x == 0:
            continue
        err = abs(taylor(kind, x, degree) - exact(kind, x))
        ref = {"value": abs(exact(kind, x)), "factor": mp.exp(-x) if kind == "expm1m" else mp.mpf(1)}[relative_to]
        worst = max(worst, err / ref)
    return worst


# (precision, function, highest power used, range, error measured relative
# to, stated bound as a power of two: at most a quarter of the unit roundoff)
CASES = [
    ("f32", "sin", 5, "0.2", "value", -26),
    ("f32", "cos", 6, "0.2", "factor", -26),
    ("f32", "expm1m", 4, "0.05", "factor", -27),
    ("f64", "sin", 9, "0.1", "value", -58),
    ("f64", "cos", 10, "0.1", "factor", -58),
    ("f64", "expm1m", 7, "0.02", "factor", -60),
]


@pytest.mark.parametrize("prec, kind, degree, rng, rel, log2_bound", CASES)
def test_series_truncation_below_a_quarter_roundoff(prec, kind, degree, rng, rel, log2_bound):
    u = U32 if prec == "f32" else U64
    bound = mp.mpf(2) ** log2_bound
    assert bound <= u / 4
    assert worst_error(kind, degree, mp.mpf(rng), rel) <= bound
    assert worst_error(kind, degree, 4 * mp.mpf(rng), rel) > bound
