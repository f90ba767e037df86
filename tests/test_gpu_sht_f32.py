"""FP32 spherical-harmonic transforms of the CUDA path (the transforms the
mixed-precision solver iterates with), through the C ABI, against the
oracle's FP64 direct sums, element by element.

Tolerance (relative to the largest output value): u (64 + 2 nside sqrt(lmax+1)),
u = 2^-24.  The second term bounds the phase drift of the FP32 Legendre
recurrence: rounding c_l to FP32 perturbs the step's frequency by ~u / tan(theta),
the errors of lmax steps add like a random walk (sqrt(lmax) u / tan(theta)),
and the ring nearest the pole has tan(theta) ~ 0.8 / nside.  The first term
covers the FP32 FFTs and sums on coarse grids."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def tol32(nside, lmax):
    return U * (64.0 + 2.0 * nside * np.sqrt(lmax + 1.0))


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


# power-of-two and Bluestein rings, ragged band limits, several CTAs per m
CASES = [(1, 2), (2, 5), (4, 8), (8, 16), (8, 7), (16, 32), (32, 64), (32, 95),
         (64, 128), (160, 320)]


@pytest.mark.parametrize("nside,lmax", CASES)
def test_alm2map_f32_matches_oracle(torch_cuda, osht, nside, lmax):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    a = rand_alm(lmax, 300 + nside + lmax)
    ref = osht.alm2map(a, nside, lmax)
    with wf.Plan(nside, lmax, np.ones(lmax + 1)) as p:
        got = p.alm2map_f32(torch.from_numpy(a).cuda()).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= tol32(nside, lmax) * np.max(np.abs(ref))


@pytest.mark.parametrize("nside,lmax", CASES)
def test_map2alm_f32_matches_oracle(torch_cuda, osht, nside, lmax):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    m = np.random.default_rng(nside * 11 + lmax).standard_normal(12 * nside * nside)
    ref = osht.map2alm(m, nside, lmax)
    with wf.Plan(nside, lmax, np.ones(lmax + 1)) as p:
        got = p.map2alm_f32(torch.from_numpy(m).cuda()).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= tol32(nside, lmax) * np.max(np.abs(ref))


@pytest.fixture(scope="module")
def full_size_case(osht):
    """Nside 1024, lmax 2048: a band-limited field, sampled pixels (the polar
    rings included) and sampled coefficients of the analysis of a white map,
    each computed one by one by the oracle."""
    from paper_1702_08852_gb300 import inputs
    nside, lmax = 1024, 2048
    npix = 12 * nside * nside
    cl = inputs.cl_spectrum(lmax, nside)
    rng = np.random.default_rng(91)
    a = inputs.random_alm(rng, np.maximum(cl, 1e-12))
    pix = np.concatenate([rng.integers(0, npix, 30),
                          [0, 3, 4, 40, npix - 1, npix // 2, 2 * nside * (nside - 1)]])
    ref = osht.alm2map_pixels(a, nside, lmax, pix)
    m = rng.standard_normal(npix)
    ls, ms = inputs.lm_of_slots(lmax)
    sel = np.concatenate([rng.integers(0, len(ls), 10), [0, inputs.nalm(lmax) - 1, 2048]])
    refb = 4 * np.pi / npix * osht.adjoint_modes(m, nside, lmax, ls[sel], ms[sel])
    return dict(nside=nside, lmax=lmax, cl=cl, a=a, pix=pix, ref=ref, m=m, sel=sel,
                refb=refb)


# the default launch variants, and those the autotuner picks on GB300 at
# Nside 1024 (the solver's timed configuration)
FULL_SIZE_TUNINGS = [None,
                     dict(ana_np=(4, 4), ana_queue=0, ana_packed=1, ana_global_acc=1),
                     dict(ana_np=(4, 4), ana_queue=0, ana_packed=1, ana_global_acc=2),
                     dict(syn_np=(1, 4), syn_packed=1), dict(syn_np=(1, 2), syn_packed=1)]


@pytest.mark.parametrize("tuning", FULL_SIZE_TUNINGS)
def test_f32_full_size_sampled(torch_cuda, full_size_case, tuning):
    """The FP32 transforms at Nside 1024 / lmax 2048 in each launch variant,
    against the oracle's sampled outputs; the measured error, relative to
    the largest output, is printed beside the bound."""
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    c = full_size_case
    with wf.Plan(c["nside"], c["lmax"], c["cl"]) as p:
        if tuning:
            p.set_tuning(**tuning)
        mp = p.alm2map_f32(torch.from_numpy(c["a"]).cuda()).cpu().numpy()
        b = p.map2alm_f32(torch.from_numpy(c["m"]).cuda()).cpu().numpy()
    tol = tol32(c["nside"], c["lmax"])
    e_syn = np.max(np.abs(mp[c["pix"]] - c["ref"])) / np.max(np.abs(mp))
    e_ana = np.max(np.abs(b[c["sel"]] - c["refb"])) / np.max(np.abs(b))
    print(f"f32 full size {tuning}: synthesis {e_syn:.3e}, analysis {e_ana:.3e}, "
          f"bound {tol:.3e}")
    assert e_syn <= tol and e_ana <= tol


VARIANTS = [dict(ana_np=(4, 2), ana_queue=0), dict(ana_np=(4, 4), ana_queue=0),
            dict(ana_np=(4, 8), ana_queue=0), dict(ana_np=(4, 16), ana_queue=0),
            dict(ana_np=(4, 4), ana_queue=1), dict(ana_np=(4, 8), ana_queue=1),
            dict(ana_np=(4, 4), ana_queue=0, ana_packed=1),
            dict(ana_np=(4, 8), ana_queue=0, ana_packed=1),
            dict(ana_np=(4, 6), ana_queue=0, ana_packed=1),
            dict(ana_np=(4, 4), ana_queue=0, ana_packed=1, ana_global_acc=1),
            dict(ana_np=(4, 6), ana_queue=0, ana_packed=1, ana_global_acc=1),
            dict(ana_np=(4, 8), ana_queue=0, ana_packed=1, ana_global_acc=2),
            dict(ana_np=(4, 6), ana_queue=0, ana_packed=1, ana_global_acc=2),
            dict(ana_np=(4, 4), ana_queue=0, ana_packed=1, ana_global_acc=2),
            dict(ana_np=(4, 8), ana_queue=0, ana_packed=1, ana_global_acc=3),
            dict(syn_np=(2, 1)), dict(syn_np=(2, 4)),
            dict(syn_np=(2, 2), syn_packed=1), dict(syn_np=(2, 4), syn_packed=1),
            dict(syn_np=(2, 2), syn_packed=2)]


@pytest.mark.parametrize("tuning", VARIANTS)
@pytest.mark.parametrize("nside,lmax", [(32, 95), (64, 128)])
def test_f32_launch_variants_match_oracle(torch_cuda, osht, tuning, nside, lmax):
    """Every launch variant of the FP32 Legendre kernels (forced through
    wf_set_tuning) against the oracle, both directions."""
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    a = rand_alm(lmax, 7 * nside + lmax)
    ref = osht.alm2map(a, nside, lmax)
    m = np.random.default_rng(lmax).standard_normal(12 * nside * nside)
    refb = osht.map2alm(m, nside, lmax)
    with wf.Plan(nside, lmax, np.ones(lmax + 1)) as p:
        p.set_tuning(**tuning)
        got = p.alm2map_f32(torch.from_numpy(a).cuda()).cpu().numpy()
        gotb = p.map2alm_f32(torch.from_numpy(m).cuda()).cpu().numpy()
        gotb2 = p.map2alm_f32(torch.from_numpy(m).cuda()).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= tol32(nside, lmax) * np.max(np.abs(ref))
    assert np.max(np.abs(gotb - refb)) <= tol32(nside, lmax) * np.max(np.abs(refb))
    assert np.array_equal(gotb, gotb2)  # deterministic, queue included


def test_tuning_report_and_bad_values(torch_cuda):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    with wf.Plan(16, 32, np.ones(33), autotune=1) as p:
        t = p.tuning()
        assert all(ms > 0 for ms in t["syn_ms"][1]) and all(ms > 0 for ms in t["ana_ms"][1])
        # FP64 has no 16-pair, queue or packed candidates
        assert all(ms == -1.0 for ms in t["ana_ms"][0][3:])
        assert all(ms == -1.0 for ms in t["syn_ms"][0][3:])
        assert t["ana_np"][1] in (2, 4, 6, 8, 16) and t["ana_queue"] in (0, 1)
        for bad in (dict(syn_np=(3, 2)), dict(ana_np=(16, 8)), dict(ana_queue=2),
                    dict(ana_np=(4, 2), ana_queue=1),
                    dict(ana_np=(4, 8), ana_queue=1, ana_packed=1),
                    dict(syn_np=(2, 1), syn_packed=1), dict(syn_np=(2, 4), syn_packed=2),
                    dict(ana_np=(4, 8), ana_packed=1, ana_global_acc=1),
                    dict(ana_np=(4, 4), ana_packed=0, ana_global_acc=2),
                    dict(ana_np=(4, 6), ana_packed=1, ana_global_acc=3),
                    dict(ana_np=(4, 4), ana_packed=0, ana_global_acc=1)):
            with pytest.raises(wf.WFError):
                p.set_tuning(**bad)
        assert p.tuning()["ana_np"] == t["ana_np"]
