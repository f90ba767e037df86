"""FP64 spherical-harmonic transforms of the CUDA path (called through the
C ABI) against the oracle's direct sums, element by element."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12   # FP64: relative to the largest output value


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_08852_gb300 import build
    build.build()
    return torch


def rand_alm(lmax, seed):
    from paper_1702_08852_gb300 import inputs
    rng = np.random.default_rng(seed)
    n = inputs.nalm(lmax)
    a = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    _, ms = inputs.lm_of_slots(lmax)
    a[ms == 0] = a[ms == 0].real
    return a


CASES = [(1, 2), (1, 1), (2, 5), (4, 8), (4, 11), (8, 16), (8, 7), (16, 32),
         (32, 64), (32, 95), (160, 320)]


@pytest.mark.parametrize("nside,lmax", CASES)
def test_alm2map_matches_oracle(torch_cuda, osht, nside, lmax):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    a = rand_alm(lmax, 100 + nside + lmax)
    ref = osht.alm2map(a, nside, lmax)
    with wf.Plan(nside, lmax, np.ones(lmax + 1)) as p:
        got = p.alm2map(torch.from_numpy(a).cuda()).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))


@pytest.mark.parametrize("nside,lmax", CASES)
def test_map2alm_matches_oracle(torch_cuda, osht, nside, lmax):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    m = np.random.default_rng(nside * 7 + lmax).standard_normal(12 * nside * nside)
    ref = osht.map2alm(m, nside, lmax)
    with wf.Plan(nside, lmax, np.ones(lmax + 1)) as p:
        got = p.map2alm(torch.from_numpy(m).cuda()).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))


def test_band_limited_sky_roundtrip_stays_exact_in_l_small(torch_cuda, osht):
    """A field with a_lm = 0 above l = 10 on a fine grid: map2alm(alm2map)
    reproduces it to the quadrature error, identical to the oracle's."""
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    nside, lmax = 32, 64
    a = rand_alm(lmax, 5)
    from paper_1702_08852_gb300 import inputs
    ls, _ = inputs.lm_of_slots(lmax)
    a[ls > 10] = 0
    ref = osht.map2alm(osht.alm2map(a, nside, lmax), nside, lmax)
    with wf.Plan(nside, lmax, np.ones(lmax + 1)) as p:
        got = p.map2alm(p.alm2map(torch.from_numpy(a).cuda())).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))


@pytest.mark.parametrize("nside", [1024])
def test_full_size_sampled(torch_cuda, osht, nside):
    """Nside 1024, lmax 2048 (the full-size workload): sampled pixels of the
    synthesis and sampled coefficients of the analysis, each computed one by
    one by the oracle's direct sum."""
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf, inputs
    lmax = 2 * nside
    cl = inputs.cl_spectrum(lmax, nside)
    rng = np.random.default_rng(77)
    a = inputs.random_alm(rng, np.maximum(cl, 1e-12))
    with wf.Plan(nside, lmax, cl) as p:
        mp = p.alm2map(torch.from_numpy(a).cuda()).cpu().numpy()
        pix = np.concatenate([rng.integers(0, 12 * nside * nside, 40),
                              [0, 1, 5, 12 * nside * nside - 1, 6 * nside * nside]])
        ref = osht.alm2map_pixels(a, nside, lmax, pix)
        scale = np.sqrt(np.mean(mp ** 2))
        assert np.max(np.abs(mp[pix] - ref)) <= 1e-11 * scale
        m = rng.standard_normal(12 * nside * nside)
        b = p.map2alm(torch.from_numpy(m).cuda()).cpu().numpy()
    ls, ms = inputs.lm_of_slots(lmax)
    sel = np.concatenate([rng.integers(0, len(ls), 10),
                          [0, inputs.nalm(lmax) - 1, 2048, 5000]])
    om = 4 * np.pi / (12 * nside * nside)
    ref = om * osht.adjoint_modes(m, nside, lmax, ls[sel], ms[sel])
    scale = np.sqrt(np.mean(np.abs(b) ** 2))
    assert np.max(np.abs(b[sel] - ref)) <= 1e-11 * scale


def tol_df64(nside, lmax):
    """Double-float Legendre step: the bound of the FP32 kernels' random-walk
    phase model with the double-float unit roundoff 2^-44 (its sums carry the
    rounding of one FP32 addition in the low part), relative to the largest
    output, floored at the FP64 tolerance."""
    return max(TOL, 2.0 ** -44 * (64.0 + 2.0 * nside * np.sqrt(lmax + 1.0)))


@pytest.mark.parametrize("nside,lmax", [(1, 2), (4, 11), (8, 16), (32, 95), (64, 128),
                                        (160, 320)])
def test_df64_transforms_match_oracle(torch_cuda, osht, nside, lmax):
    """The double-float transforms of the anchor steps against the oracle."""
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    a = rand_alm(lmax, 500 + nside + lmax)
    ref = osht.alm2map(a, nside, lmax)
    m = np.random.default_rng(3 * nside + lmax).standard_normal(12 * nside * nside)
    refb = osht.map2alm(m, nside, lmax)
    with wf.Plan(nside, lmax, np.ones(lmax + 1)) as p:
        got = p.alm2map_df64(torch.from_numpy(a).cuda()).cpu().numpy()
        gotb = p.map2alm_df64(torch.from_numpy(m).cuda()).cpu().numpy()
        gotb2 = p.map2alm_df64(torch.from_numpy(m).cuda()).cpu().numpy()
    t = tol_df64(nside, lmax)
    assert np.max(np.abs(got - ref)) <= t * np.max(np.abs(ref))
    assert np.max(np.abs(gotb - refb)) <= t * np.max(np.abs(refb))
    assert np.array_equal(gotb, gotb2)


def test_df64_full_size_sampled(torch_cuda, osht):
    """Nside 1024, lmax 2048: sampled pixels (polar rings included) and
    coefficients of the double-float transforms, one by one by the oracle."""
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf, inputs
    nside, lmax = 1024, 2048
    npix = 12 * nside * nside
    cl = inputs.cl_spectrum(lmax, nside)
    rng = np.random.default_rng(93)
    a = inputs.random_alm(rng, np.maximum(cl, 1e-12))
    with wf.Plan(nside, lmax, cl) as p:
        mp = p.alm2map_df64(torch.from_numpy(a).cuda()).cpu().numpy()
        pix = np.concatenate([rng.integers(0, npix, 30), [0, 3, 40, npix - 1, npix // 2]])
        ref = osht.alm2map_pixels(a, nside, lmax, pix)
        assert np.max(np.abs(mp[pix] - ref)) <= tol_df64(nside, lmax) * np.max(np.abs(mp))
        m = rng.standard_normal(npix)
        b = p.map2alm_df64(torch.from_numpy(m).cuda()).cpu().numpy()
    ls, ms = inputs.lm_of_slots(lmax)
    sel = np.concatenate([rng.integers(0, len(ls), 10), [0, inputs.nalm(lmax) - 1, 2048]])
    om = 4 * np.pi / npix
    ref = om * osht.adjoint_modes(m, nside, lmax, ls[sel], ms[sel])
    assert np.max(np.abs(b[sel] - ref)) <= tol_df64(nside, lmax) * np.max(np.abs(b))
