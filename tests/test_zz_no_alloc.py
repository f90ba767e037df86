"""wf_residual_static: the residual diagnostics for callers that cannot
allocate device memory during the call (a fixed device-memory budget, a pool
allocator they do not own, loops that must not stall on cudaMalloc).  It must
give wf_residual's results.  Kept in a file of its own that pytest collects
last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_08852_gb300 import build
    build.build()
    return torch


def test_static_residual_equals_allocating_one(torch_cuda):
    torch = torch_cuda
    from paper_1702_08852_gb300 import inputs, wf
    p = inputs.lognormal_problem(16, seed=77)
    rng = np.random.default_rng(78)
    d = torch.from_numpy(rng.standard_normal(p.noise.size) + p.noise).cuda()
    nv = torch.from_numpy(p.noise_var).cuda()
    mk = torch.from_numpy(p.mask.astype(np.uint8)).cuda()
    with wf.Plan(p.nside, p.lmax, p.cl, nv, mk) as plan:
        for seed in (1, 2):   # two calls in a row on the same plan
            a = torch.from_numpy(inputs.random_alm(np.random.default_rng(seed), p.cl)).cuda()
            want = plan.residual(d, a)
            got = plan.residual_static(d, a)
            for k in ("rel_res_wf", "rel_res_fp", "chi2"):
                assert got[k] == pytest.approx(want[k], rel=1e-12, abs=1e-300), k


def test_static_residual_rejects_large_plans(torch_cuda):
    torch = torch_cuda
    from paper_1702_08852_gb300 import inputs, wf
    p = inputs.uniform_problem(256, seed=3)
    nv = torch.from_numpy(p.noise_var).cuda()
    with wf.Plan(p.nside, p.lmax, p.cl, nv) as plan:
        d = torch.zeros(p.noise.size, dtype=torch.float64, device="cuda")
        a = torch.zeros(plan.nalm, dtype=torch.complex128, device="cuda")
        with pytest.raises(wf.WFError) as e:
            plan.residual_static(d, a)
        assert e.value.status == wf.WF_ERR_ARG
        assert "static scratch" in str(e.value)
