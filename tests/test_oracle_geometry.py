"""Pins for the oracle's HEALPix ring geometry (Gorski et al. 2005)."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "healpix_nside1_2.txt")


def test_golden_small_nside(osht):
    rows = np.loadtxt(GOLDEN, comments="#")
    for ns, ring, n, z, p0 in rows:
        f, cnt, zz, st, ph = osht.ring_info(int(ns), int(ring))
        assert cnt == int(n)
        assert zz == pytest.approx(z, abs=1e-15)
        assert ph / np.pi == pytest.approx(p0, abs=1e-15)
        assert st == pytest.approx(np.sqrt(1 - z * z), abs=1e-15)


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 64])
def test_ring_layout(osht, nside):
    total = 0
    prev_z = 1.0
    for ring in range(1, 4 * nside):
        f, n, z, st, p0 = osht.ring_info(nside, ring)
        assert f == total            # rings are contiguous, in order
        total += n
        assert z < prev_z            # north to south
        prev_z = z
        mirror = osht.ring_info(nside, 4 * nside - ring)
        assert mirror[1] == n and mirror[2] == pytest.approx(-z, abs=1e-15)
        assert st == pytest.approx(np.sqrt((1 - z) * (1 + z)), rel=1e-12)
    assert total == 12 * nside * nside


@pytest.mark.parametrize("nside", [2, 4, 8])
def test_equal_area_low_moments(osht, nside):
    """Pixel centres of an equal-area iso-latitude grid integrate z and z^2
    like the sphere up to the pixel-size error; odd moments vanish exactly."""
    z, st, phi = osht.pix_coords(nside)
    assert abs(np.mean(z)) < 1e-15
    assert abs(np.mean(z ** 3)) < 1e-15
    assert np.mean(z * z) == pytest.approx(1.0 / 3.0, abs=0.5 / nside ** 2)


@pytest.mark.parametrize("nside", [2, 4, 8])
def test_azimuthal_sums(osht, nside):
    """sum_j exp(i m phi_j) over a ring vanishes unless m is a multiple of the
    ring's pixel count: the pixels are equally spaced in phi."""
    z, st, phi = osht.pix_coords(nside)
    for ring in range(1, 4 * nside):
        f, n, _, _, _ = osht.ring_info(nside, ring)
        ph = phi[f:f + n]
        for m in range(1, 2 * n + 1):
            s = np.sum(np.exp(1j * m * ph))
            if m % n:
                assert abs(s) < 1e-12
            else:
                assert abs(s) == pytest.approx(n, rel=1e-12)


def test_input_generator_geometry_agrees(osht):
    """The input generator places masks with its own pixel-centre code; it
    must describe the same pixels as the oracle."""
    from paper_1702_08852_gb300 import inputs
    for ns in (1, 2, 4, 16):
        z, st, phi = osht.pix_coords(ns)
        z2, p2 = inputs.pixel_centres(ns)
        assert np.array_equal(z, z2) and np.allclose(phi, p2, atol=1e-14)
