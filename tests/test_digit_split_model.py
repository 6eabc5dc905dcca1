"""The error-free digit split behind the tensor-core trailing update (Ozaki, Ogita, Oishi and Rump, Numer.
Algorithms 59 (2012)), checked in exact arithmetic on the CPU.

Each row x of the operands is scaled by 2^-e (e the exponent of its largest magnitude) and cut into S signed
digits of B bits, x 2^-e = sum_s d_s 2^-Bs + r.  The GPU sums, per level L = s + t, the products d_s(W_i) d_t(L_j)
over the panel columns in an FP32 accumulator, and recombines the levels in 64-bit integers.  That is exact only
if every partial sum of a level is an integer below 2^24, and FP64-accurate only if the dropped digits are below
FP64 rounding.  Real updates use S = 7, B = 8 over K = 64 columns; complex ones S = 8, B = 7 over K = 128 (the real
and imaginary products of one level share an accumulator)."""
from fractions import Fraction
import math

import numpy as np
import pytest

CASES = {"real": (7, 8, 64), "complex": (8, 7, 128)}


def digits(x, S, B):
    """Row x (FP64) -> exponent e and integer digits d[S, len(x)] with x 2^-e = sum_s d_s 2^-Bs + r."""
    m = np.max(np.abs(x))
    e = math.frexp(m)[1] if m > 0 else 0
    y = np.ldexp(x, -e)
    d = np.zeros((S, x.size), dtype=np.int64)
    for s in range(S):
        y = y * 2.0 ** B
        ds = np.rint(y)
        y = y - ds
        d[s] = ds.astype(np.int64)
    return e, d


def level_sums(dw, dl, S):
    """acc_L for L = s + t (0-based, L = 0 .. S-1), exact integers."""
    acc = np.zeros(S, dtype=object)
    for s in range(S):
        for t in range(S - s):
            acc[s + t] += int(np.dot(dw[s], dl[t]))
    return acc


@pytest.mark.parametrize("case", ["real", "complex"])
def test_digit_bounds_and_worst_case_level_sums_fit_fp32(case):
    S, B, K = CASES[case]
    rng = np.random.default_rng(7)
    for _ in range(50):
        x = rng.standard_normal(64) * 2.0 ** rng.integers(-30, 30)
        _, d = digits(x, S, B)
        assert np.max(np.abs(d[0])) <= 2 ** B and np.max(np.abs(d[1:])) <= 2 ** (B - 1)
    # every digit at its bound, all products of one sign: the largest level sum any input can produce
    worst = max(K * sum((2 ** B if s == 0 else 2 ** (B - 1)) * (2 ** B if L - s == 0 else 2 ** (B - 1))
                        for s in range(L + 1)) for L in range(S))
    assert worst < 2 ** 24, worst          # exact in an FP32 accumulator (and as a float -> int conversion)


@pytest.mark.parametrize("case", ["real", "complex"])
def test_recombined_product_is_fp64_accurate(case):
    S, B, K = CASES[case]
    rng = np.random.default_rng(11)
    worst_rel = 0.0
    for trial in range(40):
        scale_w = 2.0 ** rng.integers(-6, 6, size=K)     # columns of different size, as in W = L D
        w = rng.standard_normal(K) * scale_w * 2.0 ** rng.integers(-20, 20)
        l = rng.standard_normal(K) * 2.0 ** rng.integers(-20, 20)
        ew, dw = digits(w, S, B)
        el, dl = digits(l, S, B)
        acc = level_sums(dw, dl, S)
        assert max(abs(int(a)) for a in acc) < 2 ** 24
        approx = sum(Fraction(int(acc[L])) / 2 ** (B * (L + 2)) for L in range(S)) * Fraction(2) ** (ew + el)
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(w, l))
        bound = Fraction(float(np.max(np.abs(w)))) * Fraction(float(np.max(np.abs(l))))
        worst_rel = max(worst_rel, float(abs(approx - exact) / bound))
    # within the rounding-error bound of an FP64 dot product of this length (K u max|w| max|l|, u = 2^-53); the
    # measured worst cases are about 2^-53 (real) and 2^-52 (complex), i.e. a few units of the last place
    assert worst_rel < K * 2.0 ** -53, worst_rel


def test_digits_reconstruct_the_row():
    S, B, _ = CASES["real"]
    x = np.array([1.0, -0.5, 3.0e-5, 2.0 ** -40, -1.0 + 2.0 ** -52, 0.0])
    e, d = digits(x, S, B)
    rec = [sum(Fraction(int(d[s, j])) / 2 ** (B * (s + 1)) for s in range(S)) * Fraction(2) ** e
           for j in range(x.size)]
    m = Fraction(float(np.max(np.abs(x))))
    for j in range(x.size):
        assert abs(rec[j] - Fraction(float(x[j]))) <= m * Fraction(1, 2 ** (B * S))
