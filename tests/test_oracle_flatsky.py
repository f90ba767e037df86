"""Pins for the oracle's flat-sky dual messenger (Algorithm 2 with 2-D FFTs,
the paper's Sect. 3 set-up): the uniform-noise closed form, and -- the basis
change being orthogonal here -- convergence to the Wiener filter of Eq. (2)
itself, against a dense solve and a conjugate-gradient solve."""
import numpy as np
import pytest

from paper_1702_08852_gb300 import inputs


@pytest.fixture(scope="module")
def ofs():
    from oracle import flatsky
    return flatsky


def setup(ofs, n, seed, uniform=False):
    side = np.deg2rad(10.0) * n / 512 * 8 if n < 64 else np.deg2rad(10.0)
    om = (side / n) ** 2
    ck = inputs.flat_cl(inputs.flat_mode_ell(n, side))
    rng = np.random.default_rng(seed)
    if uniform:
        nv, _ = np.full((n, n), 64.0), None
    else:
        nv, _ = inputs.flat_paper_noise(n, side_deg=np.rad2deg(side), mask_deg=np.rad2deg(side) / 2)
    s = inputs.flat_gaussian_field(rng, ck, om)
    d = s + np.sqrt(nv) * rng.standard_normal((n, n))
    return d, nv, ck, om


def test_uniform_noise_closed_form(ofs):
    d, nv, ck, om = setup(ofs, 32, 1, uniform=True)
    s, info = ofs.dual_messenger_flat(d, nv, ck, om, eps_final=1e-12)
    assert info["converged"] and info["iterations"] <= 2 * info["stages"]
    want = np.real(np.fft.ifft2(ck / (ck + 64.0 * om) * np.fft.fft2(d)))
    assert np.linalg.norm(s - want) / np.linalg.norm(want) < 1e-12


@pytest.mark.parametrize("n", [8, 16])
def test_fixed_point_is_the_wiener_filter(ofs, n):
    """Masked-square noise (10^6 N inside): the last stage's fixed point is
    the exact Wiener filter, here by a dense solve s = S (S + N)^-1 d."""
    d, nv, ck, om = setup(ofs, n, 2 + n)
    s, info = ofs.dual_messenger_flat(d, nv, ck, om, eps_final=1e-14, stop="error")
    assert info["converged"]
    want = ofs.wf_dense(d, nv, ck, om)
    assert np.linalg.norm(s - want) / np.linalg.norm(want) < 1e-9


def test_cg_matches_dense(ofs):
    d, nv, ck, om = setup(ofs, 16, 7)
    s, info = ofs.wf_cg(d, nv, ck, om, tol=1e-13)
    want = ofs.wf_dense(d, nv, ck, om)
    assert info["rel_residual"] < 1e-13
    assert np.linalg.norm(s - want) / np.linalg.norm(want) < 1e-10


def test_paper_workload_shapes(ofs):
    """512^2, L = 10 deg, 64 muK^2, central 5 deg square at 10^6 N: a quarter
    of the map masked; l of the fundamental mode 2 pi / L."""
    nv, m = inputs.flat_paper_noise(512)
    assert m.mean() == pytest.approx(0.25, abs=0.01)
    assert nv.min() == 64.0 and nv.max() == 64.0e6
    ell = inputs.flat_mode_ell(512, np.deg2rad(10.0))
    assert ell[0, 1] == pytest.approx(2 * np.pi / np.deg2rad(10.0))
    assert inputs.flat_cl(ell)[0, 0] == 0.0
