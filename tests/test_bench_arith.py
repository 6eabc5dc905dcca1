"""The arithmetic behind bench.py's roofline fields, on CPU: the trailing-update work count against a brute-force
count of the updated elements, and the roofline of each kernel class from a synthetic per-launch profile (achieved
rate = algorithmic flops / measured time, fraction = achieved / the stated peak, the dominant class chosen by
serialised time per step)."""
import types

import numpy as np
import pytest

import bench


@pytest.mark.parametrize("n", [64, 65, 130, 200, 257])
def test_ldlt_update_macs_brute_force(n):
    # every block step k1 = 64, 128, ... updates A_ij (i >= j >= k1) with 64 multiply-adds
    brute = 0
    for k1 in range(64, n, 64):
        brute += sum(1 for i in range(k1, n) for j in range(k1, i + 1)) * 64
    assert bench.ldlt_update_macs(n) == brute


def test_rooflines_from_synthetic_profile():
    n, nov = 4000, 129_600
    spec = types.SimpleNamespace(n_aux=n, n_ov=nov)
    prm = types.SimpleNamespace(n_imag=100, n_real=40)
    # four imaginary frequencies and two near-real points timed, per class (launches, total ms)
    prof_i = {"pi_tc_imag": (4, 4 * 4.5), "ldlt_update": (248, 4 * 2.0), "ldlt": (4, 99.0), "pi_prep": (5, 3.3)}
    prof_r = {"pi_tc_complex": (2, 2 * 9.0), "ldlt_update": (124, 2 * 5.0), "ldlt": (2, 77.0)}
    peaks = {"bf16_tflops": 1900.0}
    rl, shares = bench.rooflines(spec, prm, (prof_i, prof_r, 4, 2), peaks, "measured", True)
    pi_flops = n * (n + 1) / 2 * nov * 2.0
    ach = pi_flops / 4.5e-3 / 1e12
    assert rl["pi_tc_imag"]["achieved"] == pytest.approx(ach)
    assert rl["pi_tc_imag"]["frac"] == pytest.approx(ach / (1900.0 / 3))
    assert rl["pi_tc_imag"]["serialised_ms_per_step"] == pytest.approx(4.5 * 100)
    assert rl["pi_tc_complex"]["achieved"] == pytest.approx(2 * pi_flops / 9.0e-3 / 1e12)
    macs = bench.ldlt_update_macs(n)
    assert rl["oz_update_real"]["achieved"] == pytest.approx(28 * macs * 2.0 / 2.0e-3 / 1e12)
    assert rl["oz_update_real"]["frac"] == pytest.approx(28 * macs * 2.0 / 2.0e-3 / 1e12 / 1900.0)
    assert rl["oz_update_complex"]["achieved"] == pytest.approx(144 * macs * 2.0 / 5.0e-3 / 1e12)
    # the whole-factorisation class is not a share of its own parts; the shares sum to one
    assert "ldlt" not in shares
    assert sum(v["share"] for v in shares.values()) == pytest.approx(1.0)
    assert shares["pi_tc_imag"]["serialised_ms_per_step"] == pytest.approx(18.0 / 4 * 100)
    assert shares["ldlt_update"]["serialised_ms_per_step"] == pytest.approx(8.0 / 4 * 100 + 10.0 / 2 * 40)
    # the bench line's roofline is the class with the most serialised time among the tensor kernels
    # (Pi(i xi) 450 ms, Pi(z) 360, real updates 200, complex updates 200)
    assert max(rl, key=lambda k: rl[k]["serialised_ms_per_step"]) == "pi_tc_imag"
