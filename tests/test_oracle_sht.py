"""Pins for the oracle's direct synthesis Y and transpose Y^T."""
import math

import numpy as np
import pytest


def rand_alm(osht, lmax, rng):
    a = rng.standard_normal(osht.nalm(lmax)) + 1j * rng.standard_normal(osht.nalm(lmax))
    _, ms = osht.lm_arrays(lmax)
    a[ms == 0] = a[ms == 0].real
    return a


@pytest.mark.parametrize("nside,lmax", [(2, 5), (4, 8), (4, 11), (8, 16), (8, 23)])
def test_adjoint_identity(osht, nside, lmax):
    """<Y x, m> = <x, Y^T m> with the real-basis inner product."""
    rng = np.random.default_rng(nside * 100 + lmax)
    a = rand_alm(osht, lmax, rng)
    m = rng.standard_normal(osht.npix(nside))
    lhs = float(np.dot(osht.alm2map(a, nside, lmax), m))
    rhs = osht.alm_dot(a, osht.adjoint(m, nside, lmax), lmax)
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_single_modes_closed_form(osht):
    """Synthesis of one (l, m) coefficient equals the textbook Y_lm on every
    pixel: a_l0 = 1 -> Y_l0; a_lm = 1 -> 2 Re Y_lm; a_lm = i -> -2 Im Y_lm."""
    nside, lmax = 4, 2
    z, st, phi = osht.pix_coords(nside)
    pi = math.pi
    Y = {
        (0, 0): np.full_like(z, 1 / math.sqrt(4 * pi)),
        (1, 0): math.sqrt(3 / (4 * pi)) * z,
        (1, 1): -math.sqrt(3 / (8 * pi)) * st * np.exp(1j * phi),
        (2, 0): math.sqrt(5 / (16 * pi)) * (3 * z * z - 1),
        (2, 1): -math.sqrt(15 / (8 * pi)) * z * st * np.exp(1j * phi),
        (2, 2): 0.25 * math.sqrt(15 / (2 * pi)) * st * st * np.exp(2j * phi),
    }
    for (l, m), ylm in Y.items():
        for val in (1.0, 1j):
            if m == 0 and val == 1j:
                continue
            a = np.zeros(osht.nalm(lmax), dtype=complex)
            a[osht.alm_index(lmax, l, m)] = val
            s = osht.alm2map(a, nside, lmax)
            want = ylm.real if m == 0 else 2 * (val * ylm).real
            assert np.max(np.abs(s - want)) < 1e-14


def test_synthesis_against_scipy(osht):
    """A random band-limited field summed term by term with scipy's Y_lm."""
    special = pytest.importorskip("scipy.special")
    if not hasattr(special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    nside, lmax = 4, 9
    rng = np.random.default_rng(7)
    a = rand_alm(osht, lmax, rng)
    z, st, phi = osht.pix_coords(nside)
    th = np.arccos(z)
    want = np.zeros_like(z)
    for l in range(lmax + 1):
        for m in range(l + 1):
            y = special.sph_harm_y(l, m, th, phi)
            c = a[osht.alm_index(lmax, l, m)]
            want += (c * y).real if m == 0 else 2 * (c * y).real
    got = osht.alm2map(a, nside, lmax)
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))


def test_ymatrix_and_real_basis(osht):
    nside, lmax = 4, 8
    rng = np.random.default_rng(3)
    a = rand_alm(osht, lmax, rng)
    Y = osht.ymatrix(nside, lmax)
    x = osht.alm_to_real(a, lmax)
    assert np.allclose(osht.real_to_alm(x, lmax), a, rtol=0, atol=1e-15)
    assert np.dot(x, x) == pytest.approx(osht.alm_dot(a, a, lmax), rel=1e-14)
    assert np.max(np.abs(Y @ x - osht.alm2map(a, nside, lmax))) < 1e-13
    m = rng.standard_normal(osht.npix(nside))
    assert np.max(np.abs(osht.real_to_alm(Y.T @ m, lmax)
                         - osht.adjoint(m, nside, lmax))) < 1e-13


def test_selected_pixels_and_modes(osht):
    nside, lmax = 8, 16
    rng = np.random.default_rng(5)
    a = rand_alm(osht, lmax, rng)
    full = osht.alm2map(a, nside, lmax)
    pix = rng.integers(0, osht.npix(nside), 40)
    assert np.array_equal(osht.alm2map_pixels(a, nside, lmax, pix), full[pix])
    m = rng.standard_normal(osht.npix(nside))
    b = osht.adjoint(m, nside, lmax)
    ls, ms = osht.lm_arrays(lmax)
    sel = rng.integers(0, len(ls), 30)
    got = osht.adjoint_modes(m, nside, lmax, ls[sel], ms[sel])
    assert np.max(np.abs(got - b[sel])) < 1e-12


def test_constant_map_analysis(osht):
    """Omega Y^T 1 = sqrt(4 pi) e_00 plus modes whose azimuthal sums do not
    vanish (m a multiple of every ring's pixel count: only m = 0 here) -- and
    the m = 0, l > 0 part is the (nonzero) quadrature error of HEALPix."""
    nside, lmax = 8, 16
    b = osht.map2alm(np.ones(osht.npix(nside)), nside, lmax)
    assert b[0].real == pytest.approx(math.sqrt(4 * math.pi), rel=1e-14)
    _, ms = osht.lm_arrays(lmax)
    assert np.max(np.abs(b[(ms > 0) & (ms % 4 != 0)])) < 1e-13


def test_quadrature_is_not_exact(osht):
    """Omega Y^T Y is close to, but not, the identity at lmax = 2 Nside: the
    HEALPix basis change is only approximately orthogonal (the premise of the
    messenger field, Sect. 2.1, holds to this accuracy).  Recorded, not a
    pin of exactness."""
    nside, lmax = 8, 16
    Y = osht.ymatrix(nside, lmax)
    om = 4 * math.pi / osht.npix(nside)
    E = om * Y.T @ Y - np.eye(Y.shape[1])
    err = np.max(np.abs(E))
    assert 1e-4 < err < 0.2
    # a smaller band limit is integrated much better
    Y2 = osht.ymatrix(nside, 8)
    err2 = np.max(np.abs(om * Y2.T @ Y2 - np.eye(Y2.shape[1])))
    assert err2 < err
