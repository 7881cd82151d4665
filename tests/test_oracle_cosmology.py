"""Pins for the oracle's quadrature and cosmology (Eq. 1, flat LCDM).

Closed forms: Om = 0 (de Sitter, I = z) and Om = 1 (Einstein-de Sitter,
I = 2 (1 - (1+z)^-1/2)); the low-redshift Hubble law with deceleration
q0 = 3 Om / 2 - 1; the exactness degree of the Gauss-Kronrod rule.
"""
import math

import numpy as np
import pytest


@pytest.mark.parametrize("k", range(0, 25))
def test_kronrod15_exact_to_degree_22(orc, k):
    # symmetric rule: odd powers vanish; even powers exact up to 3 * 7 + 1 = 22
    exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
    got = orc.rule_poly(k, 0)
    if k <= 22 or k % 2 == 1:
        assert abs(got - exact) < 1e-15
    else:
        assert abs(got - exact) > 1e-12


@pytest.mark.parametrize("k", range(0, 17))
def test_gauss7_exact_to_degree_13(orc, k):
    exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
    got = orc.rule_poly(k, 1)
    if k <= 13 or k % 2 == 1:
        assert abs(got - exact) < 1e-15
    else:
        assert abs(got - exact) > 1e-8


@pytest.mark.parametrize("z", [1e-4, 0.05, 0.5, 1.0, 2.0, 5.0])
def test_de_sitter_closed_form(orc, z):
    assert orc.D(z, 0.0) == pytest.approx(z * (1 + z), rel=1e-13)
    assert orc.Dprime(z, 0.0) == pytest.approx(1 + 2 * z, rel=1e-13)


@pytest.mark.parametrize("z", [1e-4, 0.05, 0.5, 1.0, 2.0, 5.0])
def test_einstein_de_sitter_closed_form(orc, z):
    I = 2.0 * (1.0 - (1.0 + z) ** -0.5)
    assert orc.I(z, 1.0) == pytest.approx(I, rel=1e-13)
    assert orc.D(z, 1.0) == pytest.approx((1 + z) * I, rel=1e-13)
    assert orc.E(z, 1.0) == pytest.approx((1 + z) ** 1.5, rel=1e-15)


@pytest.mark.parametrize("x", [1e-3, 0.1, 0.7, 1.9, 3.3])
def test_inverse_closed_forms(orc, x):
    assert orc.z_of_x(x, 0.0, 20.0) == pytest.approx(0.5 * (math.sqrt(1 + 4 * x) - 1), rel=1e-12)
    u = ((1.0 + math.sqrt(1.0 + 2.0 * x)) / 2.0) ** 2
    assert orc.z_of_x(x, 1.0, 20.0) == pytest.approx(u - 1.0, rel=1e-12)


@pytest.mark.parametrize("om", [0.1, 0.3, 0.5])
@pytest.mark.parametrize("z", [1e-3, 1e-2])
def test_low_redshift_series(orc, om, z):
    # D(z) = z + (1 - q0) z^2 / 2 + O(z^3), q0 = 3 Om / 2 - 1
    q0 = 1.5 * om - 1.0
    assert abs(orc.D(z, om) - (z + 0.5 * (1 - q0) * z * z)) < 2.0 * z ** 3


@pytest.mark.parametrize("om", [0.1, 0.3, 0.5])
@pytest.mark.parametrize("x", [0.05, 0.9, 2.5])
def test_root_round_trip_and_derivative(orc, om, x):
    z = orc.z_of_x(x, om, 10.0)
    assert orc.D(z, om) == pytest.approx(x, rel=1e-13)
    h = 1e-5
    fd = (orc.D(z + h, om) - orc.D(z - h, om)) / (2 * h)
    assert orc.Dprime(z, om) == pytest.approx(fd, rel=1e-8)


def test_distance_monotone_and_bounded(orc):
    zs = np.linspace(0.0, 2.0, 41)
    for om in (0.1, 0.3, 0.5):
        d = np.array([orc.D(z, om) for z in zs])
        assert np.all(np.diff(d) > 0)
        assert np.all(d <= zs * (1 + zs) + 1e-15)   # E >= 1 for z >= 0
