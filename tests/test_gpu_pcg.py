"""The preconditioned conjugate-gradient Wiener filter (App. C) on the CUDA
path, through the C ABI, against the oracle's PCG and the dense exact
Wiener filter (Eq. 2): both stop rules, the restarts, and the status when
the iteration limit is hit."""
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


def problem(osht, kind, nside, seed, **kw):
    from paper_1702_08852_gb300 import inputs
    if kind == "lognormal":
        p = inputs.lognormal_problem(nside, seed=seed, **kw)
    else:
        p = inputs.scan_problem(nside, seed=seed, **kw)
    return p, p.data(osht.alm2map(p.alm_true, p.nside, p.lmax))


def gpu_pcg(torch, p, d, **kw):
    from paper_1702_08852_gb300 import wf
    nv = torch.from_numpy(p.noise_var).cuda()
    mk = torch.from_numpy(p.mask.astype(np.uint8)).cuda()
    with wf.Plan(p.nside, p.lmax, p.cl, nv, mk) as plan:
        alm, mp, st = plan.pcg(torch.from_numpy(d).cuda(), **kw)
        return alm.cpu().numpy(), mp.cpu().numpy(), st


def rel(osht, a, b, lmax):
    return osht.alm_norm(a - b, lmax) / osht.alm_norm(b, lmax)


@pytest.mark.parametrize("nside,kind,seed", [(8, "lognormal", 3), (16, "scan", 4)])
def test_residual_rule_matches_oracle_and_dense_wf(torch_cuda, osht, odm, nside, kind, seed):
    from paper_1702_08852_gb300 import wf
    kw = {"discs": 10, "disc_radius_deg": 5.0} if kind == "scan" else {}
    p, d = problem(osht, kind, nside, seed, **kw)
    xo, info = odm.pcg_wf(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, tol=1e-10)
    alm, mp, st = gpu_pcg(torch_cuda, p, d, tol=1e-10, stop_rule=wf.WF_PCG_STOP_RESIDUAL)
    assert st["converged"] == 1 and st["fp_residual"] < 1e-10
    assert abs(st["iterations"] - info["iterations"]) <= 1
    assert rel(osht, alm, xo, p.lmax) < 1e-8
    if nside <= 8:
        xw = odm.wf_exact_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d)
        assert rel(osht, alm, xw, p.lmax) < 1e-8
    sref = osht.alm2map(alm, p.nside, p.lmax)
    assert np.max(np.abs(mp - sref)) <= 1e-10 * np.max(np.abs(sref))


def test_cauchy_rule_matches_oracle(torch_cuda, osht, odm):
    """App. C's criterion ||z_{i+1} - z_i|| / ||z_{i+1}|| < eps."""
    from paper_1702_08852_gb300 import wf
    p, d = problem(osht, "lognormal", 8, 13)
    xo, info = odm.pcg_wf(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, tol=1e-6,
                          stop="cauchy")
    alm, _, st = gpu_pcg(torch_cuda, p, d, tol=1e-6, stop_rule=wf.WF_PCG_STOP_CAUCHY)
    assert st["converged"] == 1 and st["final_cauchy"] < 1e-6
    assert abs(st["iterations"] - info["iterations"]) <= 1
    assert rel(osht, alm, xo, p.lmax) < 1e-7


def test_restarts_match_oracle(torch_cuda, osht, odm):
    """Restarting every 7 iterations (r recomputed from z) as the oracle does."""
    from paper_1702_08852_gb300 import wf
    p, d = problem(osht, "lognormal", 8, 17)
    xo, info = odm.pcg_wf(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, tol=1e-9,
                          restart=7)
    alm, _, st = gpu_pcg(torch_cuda, p, d, tol=1e-9, stop_rule=wf.WF_PCG_STOP_RESIDUAL,
                         restart=7)
    assert abs(st["iterations"] - info["iterations"]) <= 1
    assert rel(osht, alm, xo, p.lmax) < 1e-7


def test_iteration_limit_reports_not_converged(torch_cuda, osht):
    from paper_1702_08852_gb300 import wf
    p, d = problem(osht, "lognormal", 8, 5)
    alm, _, st = gpu_pcg(torch_cuda, p, d, tol=1e-14, max_iter=3)
    assert st["status"] == wf.WF_ERR_NOT_CONVERGED and st["iterations"] == 3
    assert np.all(np.isfinite(alm))
