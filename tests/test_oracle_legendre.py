"""Pins for the oracle's normalised associated Legendre functions: closed
forms, an independent library evaluation, exact quadrature orthonormality and
an arbitrary-precision check of the deep-underflow path."""
import math

import numpy as np
import pytest


def closed_forms(z):
    st = math.sqrt((1 - z) * (1 + z))
    pi = math.pi
    return {
        (0, 0): 1 / math.sqrt(4 * pi),
        (1, 0): math.sqrt(3 / (4 * pi)) * z,
        (1, 1): -math.sqrt(3 / (8 * pi)) * st,
        (2, 0): math.sqrt(5 / (16 * pi)) * (3 * z * z - 1),
        (2, 1): -math.sqrt(15 / (8 * pi)) * z * st,
        (2, 2): 0.25 * math.sqrt(15 / (2 * pi)) * st * st,
    }


@pytest.mark.parametrize("z", [0.93, 0.2, -0.55, 1 - 1e-9])
def test_closed_forms(osht, z):
    lam = osht.lambda_all(2, z, math.sqrt((1 - z) * (1 + z)))
    for (l, m), v in closed_forms(z).items():
        assert lam[osht.alm_index(2, l, m)] == pytest.approx(v, rel=1e-14, abs=1e-300)


@pytest.mark.parametrize("z", [0.3, -0.77, 0.9995])
def test_against_scipy(osht, z):
    special = pytest.importorskip("scipy.special")
    if not hasattr(special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    lmax = 60
    lam = osht.lambda_all(lmax, z, math.sqrt((1 - z) * (1 + z)))
    ls, ms = osht.lm_arrays(lmax)
    ref = special.sph_harm_y(ls, ms, math.acos(z), 0.0).real
    assert np.max(np.abs(lam - ref)) < 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("m", [0, 1, 5, 17])
def test_quadrature_orthonormality(osht, m):
    """2 pi int lam_lm lam_l'm dz = delta_ll' ; Gauss-Legendre with lmax+1
    nodes integrates these degree <= 2 lmax polynomials exactly."""
    lmax = 24
    x, w = np.polynomial.legendre.leggauss(lmax + 1)
    tab = np.array([osht.lambda_m(lmax, m, z, math.sqrt((1 - z) * (1 + z)))
                    for z in x])                      # (nodes, l-m)
    gram = 2 * math.pi * (tab * w[:, None]).T @ tab
    assert np.max(np.abs(gram - np.eye(lmax + 1 - m))) < 1e-13


@pytest.mark.parametrize("l,m,z", [(1500, 1200, 0.2), (2048, 1900, 0.05),
                                   (2048, 3, -0.31)])
def test_high_order_against_mpmath(osht, l, m, z):
    """Large m with a seed far below the double range (the recurrence must
    carry the exponent) against a 60-digit evaluation."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    st = math.sqrt((1 - z) * (1 + z))
    lam = osht.lambda_m(l, m, z, st)[l - m]
    zz = mpmath.mpf(z)
    norm = mpmath.sqrt((2 * l + 1) / (4 * mpmath.pi)
                       * mpmath.factorial(l - m) / mpmath.factorial(l + m))
    ref = norm * mpmath.legenp(l, m, zz, type=2, maxprec=200000,
                                maxterms=10 ** 6)
    ref = float(ref)
    if abs(ref) < 1e-300:
        assert abs(lam) < 1e-290
    else:
        assert lam == pytest.approx(ref, rel=1e-11)


def test_seed_far_below_double_range(osht):
    """lam_mm for m = 1200 at sin(theta) = 0.5 is ~1e-361: it is stored as 0,
    while the recurrence (carrying the exponent) still reaches the O(0.1)
    values past the turning point l ~ m / sin(theta)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 80
    m, st = 1200, 0.5
    z = math.sqrt(1 - st * st)
    lmax = 2600
    lam = osht.lambda_m(lmax, m, z, st)
    assert lam[0] == 0.0
    for l in (2450, 2600):
        norm = mpmath.sqrt((2 * l + 1) / (4 * mpmath.pi)
                           * mpmath.factorial(l - m) / mpmath.factorial(l + m))
        ref = float(norm * mpmath.legenp(l, m, mpmath.mpf(z), type=2,
                                         maxprec=200000, maxterms=10 ** 6))
        assert abs(ref) > 1e-3
        assert lam[l - m] == pytest.approx(ref, rel=1e-10)
