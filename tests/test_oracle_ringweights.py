"""Ring-weighted quadrature (oracle/ringweights.py): pins, and the measured
reason the weighted map2alm is not on the GPU path.

Pins: the weighted pixel sum integrates every Legendre polynomial up to the
chosen degree exactly (int P_l dOmega = 4 pi delta_l0), the first even degree
above it is not integrated exactly (so the pin is not vacuous), and for
degree 0 the weights are all 1 (the plain sum already integrates a
constant).  Finding: at lmax = 2 Nside the weights barely move
Omega Y^T W Y away from its error against the identity.  That error is
mostly azimuthal aliasing in the polar rings (n = 4i points for m up to
2 Nside), which no per-ring weight can remove, so the messenger's quadrature
gap stays."""
import numpy as np
import pytest
from scipy.special import eval_legendre


@pytest.fixture(scope="module")
def orw(osht):
    from oracle import ringweights
    return ringweights


@pytest.mark.parametrize("nside,lq", [(4, 8), (8, 16), (8, 24), (16, 32)])
def test_weights_integrate_legendre_exactly(osht, orw, nside, lq):
    w = orw.ring_weights(nside, lq)
    wp = orw.pixel_weights(nside, w)
    z, _, _ = osht.pix_coords(nside)
    om = 4.0 * np.pi / osht.npix(nside)
    for l in range(lq + 1):
        q = om * np.sum(wp * eval_legendre(l, z))
        assert abs(q - (4.0 * np.pi if l == 0 else 0.0)) < 1e-12, (l, q)
    # the first even degree above lq is not integrated exactly
    q = om * np.sum(wp * eval_legendre(lq + 2, z))
    assert abs(q) > 1e-10


def test_degree_zero_weights_are_one(orw):
    for nside in (2, 4, 8):
        assert np.allclose(orw.ring_weights(nside, 0), 1.0, atol=1e-14, rtol=0)


def test_weights_do_not_remove_the_gap_at_lmax_2nside(osht, orw):
    nside, lmax = 8, 16
    Y = osht.ymatrix(nside, lmax)
    om = 4.0 * np.pi / osht.npix(nside)
    eye = np.eye(Y.shape[1])
    plain = om * Y.T @ Y - eye
    for lq in (lmax, 3 * lmax // 2):
        wp = orw.pixel_weights(nside, orw.ring_weights(nside, lq))
        weighted = om * Y.T @ (wp[:, None] * Y) - eye
        # no more than a 10 % change of either norm of the error
        assert np.linalg.norm(weighted) > 0.9 * np.linalg.norm(plain)
        assert np.abs(weighted).max() > 0.9 * np.abs(plain).max()
