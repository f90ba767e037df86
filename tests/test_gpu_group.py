"""Grouped transforms (wf_map2alm_group / wf_alm2map_group): the Legendre
step of several maps that share a geometry as one tensor-core product per m
(3xTF32 split products, FP32 accumulation), through the C ABI.

Against the oracle's FP64 direct sums, map by map and element by element,
with the FP32 transforms' tolerance u (64 + 2 nside sqrt(lmax+1)), u = 2^-24,
relative to the largest output (the table is FP64-exact to TF32 hi + lo, the
products carry ~2^-21 relative, the ring FFTs are FP32).  Cases cover one
and several 128-row l tiles per (m, parity), one and several 128-pair tiles
(ragged last tile), ragged K chunks, power-of-two and Bluestein rings, odd
lmax, one map, groups that pad N, and more maps than one launch takes."""
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


def rand_alms(lmax, n, seed):
    from paper_1702_08852_gb300 import inputs
    rng = np.random.default_rng(seed)
    k = inputs.nalm(lmax)
    a = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    _, ms = inputs.lm_of_slots(lmax)
    a[:, ms == 0] = a[:, ms == 0].real
    # maps of very different amplitude in one group
    return a * np.logspace(-3, 3, n)[:, None]


CASES = [(1, 2, 1), (2, 5, 3), (4, 8, 2), (8, 7, 9), (8, 16, 1), (16, 32, 4),
         (32, 95, 3), (80, 160, 2), (96, 287, 2)]


@pytest.mark.parametrize("nside,lmax,nmaps", CASES)
def test_alm2map_group_matches_oracle(torch_cuda, osht, nside, lmax, nmaps):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    a = rand_alms(lmax, nmaps, 500 + nside + lmax)
    with wf.Plan(nside, lmax, np.ones(lmax + 1)) as p:
        got = p.alm2map_group(torch.from_numpy(a).cuda()).cpu().numpy()
    for b in range(nmaps):
        ref = osht.alm2map(a[b], nside, lmax)
        err = np.max(np.abs(got[b] - ref)) / np.max(np.abs(ref))
        assert err <= tol32(nside, lmax), (b, err)


@pytest.mark.parametrize("nside,lmax,nmaps", CASES)
def test_map2alm_group_matches_oracle(torch_cuda, osht, nside, lmax, nmaps):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    rng = np.random.default_rng(nside * 13 + lmax)
    m = rng.standard_normal((nmaps, 12 * nside * nside)) * np.logspace(2, -2, nmaps)[:, None]
    with wf.Plan(nside, lmax, np.ones(lmax + 1)) as p:
        got = p.map2alm_group(torch.from_numpy(m).cuda()).cpu().numpy()
    for b in range(nmaps):
        ref = osht.map2alm(m[b], nside, lmax)
        err = np.max(np.abs(got[b] - ref)) / np.max(np.abs(ref))
        assert err <= tol32(nside, lmax), (b, err)


def test_group_more_maps_than_one_launch(torch_cuda, osht):
    """131 maps: a launch of 128 and one of 3, each map checked against the
    per-map FP64 GPU transform, three of them against the oracle too."""
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    nside, lmax, n = 8, 16, 131
    a = rand_alms(lmax, n, 77)
    rng = np.random.default_rng(78)
    m = rng.standard_normal((n, 12 * nside * nside))
    with wf.Plan(nside, lmax, np.ones(lmax + 1)) as p:
        ad, md = torch.from_numpy(a).cuda(), torch.from_numpy(m).cuda()
        mg = p.alm2map_group(ad).cpu().numpy()
        ag = p.map2alm_group(md).cpu().numpy()
        mf = np.stack([p.alm2map(ad[b]).cpu().numpy() for b in range(n)])
        af = np.stack([p.map2alm(md[b]).cpu().numpy() for b in range(n)])
        st = p.group_stats()
    tol = tol32(nside, lmax)
    for b in range(n):
        assert np.max(np.abs(mg[b] - mf[b])) <= tol * np.max(np.abs(mf[b]))
        assert np.max(np.abs(ag[b] - af[b])) <= tol * np.max(np.abs(af[b]))
    for b in (0, 127, 130):
        ref = osht.alm2map(a[b], nside, lmax)
        assert np.max(np.abs(mg[b] - ref)) <= tol * np.max(np.abs(ref))
    assert st["launches"] == 4 and st["gflop"] > 0 and st["gbytes"] > 0


def test_group_zero_maps_and_errors(torch_cuda):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    with wf.Plan(4, 8, np.ones(9)) as p:
        e = torch.empty((0, p.nalm), dtype=torch.complex128, device="cuda")
        assert p.alm2map_group(e).shape == (0, p.npix)
        L = wf.lib()
        assert L.wf_alm2map_group(p.handle, -1, None, None) == wf.WF_ERR_ARG
        assert L.wf_map2alm_group(p.handle, 2, None, None) == wf.WF_ERR_ARG
        assert L.wf_map2alm_group(p.handle, 0, None, None) == wf.WF_OK


def test_group_at_scale_matches_fp64(torch_cuda):
    """Nside 256, lmax 512 (the group size of a 64-map batch): each of 64
    maps against the per-map FP64 GPU transforms, both directions on the
    same FP64 inputs; the grouped path's relative L2 errors are printed
    beside those of the per-map FP32 transforms."""
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf, inputs
    nside, lmax, n = 256, 512, 64
    cl = inputs.cl_spectrum(lmax, nside)
    rng = np.random.default_rng(5)
    a = np.stack([inputs.random_alm(rng, np.maximum(cl, 1e-12)) for _ in range(n)])
    a *= rng.uniform(0.5, 2.0, n)[:, None]
    rel = lambda x, y: float(torch.linalg.norm(x - y) / torch.linalg.norm(y))
    with wf.Plan(nside, lmax, cl) as p:
        ad = torch.from_numpy(a).cuda()
        mf = torch.stack([p.alm2map(ad[b]) for b in range(n)])
        af = torch.stack([p.map2alm(mf[b]) for b in range(n)])
        mg = p.alm2map_group(ad)
        ag = p.map2alm_group(mf)
        es = [rel(mg[b], mf[b]) for b in range(n)]
        ea = [rel(ag[b], af[b]) for b in range(n)]
        es32 = [rel(p.alm2map_f32(ad[b]), mf[b]) for b in range(0, n, 8)]
        ea32 = [rel(p.map2alm_f32(mf[b]), af[b]) for b in range(0, n, 8)]
        for b in range(n):
            assert float((mg[b] - mf[b]).abs().max()) <= tol32(nside, lmax) * float(mf[b].abs().max())
    print(f"Nside 256 rel L2, grouped: synthesis {max(es):.2e}, analysis {max(ea):.2e}; "
          f"per-map FP32: synthesis {max(es32):.2e}, analysis {max(ea32):.2e}")
    assert max(es) < 1e-5 and max(ea) < 1e-5
