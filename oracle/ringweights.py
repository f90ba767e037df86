"""Ring weights for the HEALPix quadrature of map2alm.  Test infrastructure
only (see oracle/__init__.py).  Plain FP64 numpy.

App. C's comparison method needs the exact adjoint, but the messenger's
basis change uses Omega Y^T as the inverse of Y (Sect. 2.2 moved to the
sphere).  Its error is the quadrature gap between the messenger's fixed
point and Eq. (2).  A ring-weighted analysis Omega Y^T W, with one weight
per iso-latitude ring (north and south alike), is the usual way to shrink
the latitude part of that error.  The weights here are the minimum-norm
correction of w = 1 that makes the weighted ring sum integrate the even
Legendre polynomials exactly up to degree lq:

    sum_k m_k w_k P_l(z_k) = Npix delta_l0,   l = 0, 2, ..., lq,

where k runs over ring pairs with z_k >= 0 and m_k is the pair's pixel
count (2 n_k, or n_k for the equator ring).  Odd degrees integrate to zero
by the north/south symmetry.  When there are more constraints than rings,
lstsq gives the least-squares weights.
"""
import numpy as np
from scipy.special import eval_legendre

from . import sht


def ring_pairs(nside):
    """z >= 0 and pixel count m_k of each ring pair (equator ring alone)."""
    nr = 2 * nside
    z = np.empty(nr)
    m = np.empty(nr)
    for k in range(nr):
        _, n, zz, _, _ = sht.ring_info(nside, k + 1)
        z[k] = zz
        m[k] = 2 * n if k < nr - 1 else n
    return z, m


def ring_weights(nside, lq):
    """Weights w_k (one per ring pair, north to equator) exact for even
    Legendre polynomials up to degree lq."""
    z, m = ring_pairs(nside)
    ls = np.arange(0, lq + 1, 2)
    A = np.stack([m * eval_legendre(l, z) for l in ls])
    b = np.zeros(len(ls))
    b[0] = float(sht.npix(nside))
    corr, *_ = np.linalg.lstsq(A, b - A @ np.ones(len(z)), rcond=None)
    return 1.0 + corr


def pixel_weights(nside, w):
    """The ring weight of every pixel (RING order)."""
    z, _, _ = sht.pix_coords(nside)
    zr, _ = ring_pairs(nside)
    out = np.empty_like(z)
    az = np.abs(z)
    for k, zk in enumerate(zr):
        out[np.isclose(az, zk, rtol=0.0, atol=1e-12)] = w[k]
    return out
