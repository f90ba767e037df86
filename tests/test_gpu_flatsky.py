"""The flat-sky dual messenger (Algorithm 2 with 2-D FFTs, the paper's
Sect. 3 set-up) on the CUDA path, through the C ABI, against the oracle:
the iteration trace and result under the paper's Cauchy rule, the exact
Wiener filter of Eq. (2) at the converged fixed point (dense solve), and
the uniform-noise closed form."""
import numpy as np
import pytest

from paper_1702_08852_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_08852_gb300 import build
    build.build()
    return torch


@pytest.fixture(scope="module")
def ofs():
    from oracle import flatsky
    return flatsky


def setup(ofs, n, seed, side_deg=10.0, uniform=False):
    side = np.deg2rad(side_deg)
    om = (side / n) ** 2
    ck = inputs.flat_cl(inputs.flat_mode_ell(n, side))
    rng = np.random.default_rng(seed)
    if uniform:
        nv = np.full((n, n), 64.0)
    else:
        nv, _ = inputs.flat_paper_noise(n, side_deg=side_deg, mask_deg=side_deg / 2)
    s = inputs.flat_gaussian_field(rng, ck, om)
    return s + np.sqrt(nv) * rng.standard_normal((n, n)), nv, ck, om


def gpu(torch, n, om, ck, nv, d, **opts):
    from paper_1702_08852_gb300 import wf
    with wf.FlatPlan(n, om, ck, torch.from_numpy(nv).cuda(), **opts) as fp:
        s, st = fp.solve(torch.from_numpy(d).cuda())
        return s.cpu().numpy(), st, fp.trace()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n,side", [(32, 1.25), (64, 2.5), (128, 10.0)])
def test_cauchy_rule_follows_the_oracle(torch_cuda, ofs, n, side):
    """eps = 1e-6: the oracle's stage lengths (+-1) and result."""
    d, nv, ck, om = setup(ofs, n, n + 1, side_deg=side)
    otr = []
    so, info = ofs.dual_messenger_flat(d, nv, ck, om, eps_final=1e-6, trace=otr)
    s, st, tr = gpu(torch_cuda, n, om, ck, nv, d, eps_final=1e-6)
    assert st["converged"] == 1 and info["converged"]
    no = np.bincount([k for k, _, _, _ in otr])
    ng = np.bincount(np.asarray(tr["stage"]))
    assert len(no) == len(ng) and np.all(np.abs(ng.astype(int) - no.astype(int)) <= 1)
    assert rel(s, so) < 1e-8


@pytest.mark.parametrize("n", [8, 16])
def test_fixed_point_is_the_wiener_filter(torch_cuda, ofs, n):
    d, nv, ck, om = setup(ofs, n, 3 * n, side_deg=n * 10.0 / 64)
    s, st, _ = gpu(torch_cuda, n, om, ck, nv, d, eps_final=1e-14, stop_rule=1)
    assert st["converged"] == 1
    assert rel(s, ofs.wf_dense(d, nv, ck, om)) < 1e-9


def test_uniform_noise_closed_form(torch_cuda, ofs):
    d, nv, ck, om = setup(ofs, 64, 5, uniform=True)
    s, st, _ = gpu(torch_cuda, 64, om, ck, nv, d, eps_final=1e-12)
    want = np.real(np.fft.ifft2(ck / (ck + 64.0 * om) * np.fft.fft2(d)))
    assert st["iterations"] <= 2 * st["stages"]
    assert rel(s, want) < 1e-12


def test_plan_rejects_bad_arguments(torch_cuda):
    from paper_1702_08852_gb300 import wf
    nv = torch_cuda.ones(100, dtype=torch_cuda.float64, device="cuda")
    with pytest.raises(wf.WFError):
        wf.FlatPlan(10, 1e-6, np.ones(100), nv)          # not a power of two
    nv = torch_cuda.ones(64, dtype=torch_cuda.float64, device="cuda")
    ck = np.ones(64)
    ck[3] = -1.0
    with pytest.raises(wf.WFError):
        wf.FlatPlan(8, 1e-6, ck, nv)                      # negative C
    nv[5] = 0.0
    with pytest.raises(wf.WFError):
        wf.FlatPlan(8, 1e-6, np.ones(64), nv)            # zero variance
