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


@pytest.mark.parametrize("om", [0.0, 1.0])
def test_sample_cells_closed_forms(orc, synth, om):
    # the per-sample grid cell and position come from the closed-form inverses at
    # Om = 0 (z = (sqrt(1 + 4x) - 1)/2) and Om = 1 (z = ((1 + sqrt(1 + 2x))/2)^2 - 1),
    # with x = d_L H0 / c; cells are the floor of the position, -1 where d_L <= 0 or
    # z > z_max, and z = z_max lies in the last cell
    lam = synth.FIDUCIAL.copy()
    lam[1] = om
    nz, zmax, c = 512, 2.0, 299792.458
    rng = np.random.default_rng(3)
    dl = rng.uniform(-500.0, 4.0e4, 4000).astype(np.float32)
    x = dl.astype(np.float64) * lam[0] / c
    if om == 0.0:
        z = 0.5 * (np.sqrt(1.0 + 4.0 * np.maximum(x, 0.0)) - 1.0)
    else:
        z = ((1.0 + np.sqrt(1.0 + 2.0 * np.maximum(x, 0.0))) / 2.0) ** 2 - 1.0
    pos_cf = z * (nz - 1) / zmax
    cell, pos = orc.sample_cells(lam, dl, nz, zmax)
    inside = (dl > 0) & (z <= zmax)
    assert np.array_equal(cell >= 0, inside)
    assert np.all(np.isnan(pos[~inside]))
    np.testing.assert_allclose(pos[inside], pos_cf[inside], rtol=1e-12, atol=1e-10)
    want = np.minimum(np.floor(pos_cf[inside]), nz - 2).astype(np.int32)
    near = np.abs(pos_cf[inside] - np.round(pos_cf[inside])) < 1e-8   # no claim at the node itself
    assert np.array_equal(cell[inside][~near], want[~near])
    # a distance that maps exactly to z_max lies in the last cell
    d_max = orc.D(zmax, om) * c / lam[0]
    cm, _ = orc.sample_cells(lam, np.array([np.nextafter(np.float32(d_max), np.float32(0))], np.float32), nz, zmax)
    assert cm[0] == nz - 2
