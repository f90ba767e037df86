"""The standard messenger (Algorithm 1, Sect. 2.1) on the CUDA path, through
the C ABI (opts.method = WF_METHOD_MESSENGER), against the oracle's
Algorithm 1: its iteration trace under the paper's Cauchy rule, its
converged fixed point, the uniform-noise closed form, and the mixed-precision
path against the FP64 one."""
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


@pytest.fixture(scope="module")
def omsg():
    from oracle import messenger
    return messenger


def problem(osht, kind, nside, seed, **kw):
    from paper_1702_08852_gb300 import inputs
    if kind == "lognormal":
        p = inputs.lognormal_problem(nside, seed=seed, **kw)
    elif kind == "scan":
        p = inputs.scan_problem(nside, seed=seed, **kw)
    else:
        p = inputs.uniform_problem(nside, seed=seed, **kw)
    return p, p.data(osht.alm2map(p.alm_true, p.nside, p.lmax))


def gpu_solve(torch, p, d, **opts):
    from paper_1702_08852_gb300 import wf
    nv = torch.from_numpy(p.noise_var).cuda()
    mk = torch.from_numpy(p.mask.astype(np.uint8)).cuda()
    with wf.Plan(p.nside, p.lmax, p.cl, nv, mk, method=wf.WF_METHOD_MESSENGER, **opts) as pl:
        alm, mp, st = pl.solve(torch.from_numpy(d).cuda())
        return alm.cpu().numpy(), mp.cpu().numpy(), st, pl.trace()


def rel(osht, a, b, lmax):
    return osht.alm_norm(a - b, lmax) / osht.alm_norm(b, lmax)


@pytest.mark.parametrize("nside,seed", [(8, 41), (16, 42)])
def test_cauchy_rule_follows_the_oracle(torch_cuda, osht, omsg, nside, seed):
    """Paper's criterion (eps = 1e-6, three-step tolerances, lambda from 1e4
    by 3/4): the FP64 CUDA path takes the oracle's stage lengths and result."""
    p, d = problem(osht, "lognormal", nside, seed)
    otr = []
    xo, info = omsg.standard_messenger(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d,
                                       eps_final=1e-6, trace=otr)
    alm, mp, st, tr = gpu_solve(torch_cuda, p, d, eps_final=1e-6)
    assert st["converged"] == 1 and info["converged"]
    no = np.bincount([k for k, _, _ in otr])
    ng = np.bincount(np.asarray(tr["stage"]))
    assert np.all(np.abs(ng.astype(int) - no.astype(int)) <= 1), (ng, no)
    assert rel(osht, alm, xo, p.lmax) < 1e-8
    # the lambda sequence: xi / alpha
    lam = np.asarray(tr["xi"]) / st["alpha"]
    assert lam[0] == pytest.approx(1e4) and lam[-1] == 1.0


@pytest.mark.parametrize("nside,kind,seed", [(8, "lognormal", 3), (8, "scan", 4)])
def test_converges_to_the_dense_fixed_point(torch_cuda, osht, omsg, nside, kind, seed):
    kw = {"discs": 5, "disc_radius_deg": 10.0} if kind == "scan" else {}
    p, d = problem(osht, kind, nside, seed, **kw)
    alm, mp, st, _ = gpu_solve(torch_cuda, p, d, eps_final=1e-13, stop_rule=1)
    assert st["converged"] == 1
    ref = omsg.messenger_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 1.0)
    assert rel(osht, alm, ref, p.lmax) < 1e-10


def test_uniform_noise_closed_form(torch_cuda, osht):
    p, d = problem(osht, "uniform", 8, 2)
    alm, _, st, _ = gpu_solve(torch_cuda, p, d, eps_final=1e-12)
    om = 4 * np.pi / osht.npix(p.nside)
    ls, _ = osht.lm_arrays(p.lmax)
    want = (p.cl / (p.cl + p.noise_var[0] * om))[ls] * osht.map2alm(d, p.nside, p.lmax)
    assert st["iterations"] <= 2 * st["stages"]
    assert rel(osht, alm, want, p.lmax) < 1e-12


@pytest.mark.parametrize("nside,kind,seed", [(16, "lognormal", 8), (32, "scan", 9)])
def test_mixed_messenger_reproduces_fp64(torch_cuda, osht, nside, kind, seed):
    """The mixed-precision path (default anchoring) takes the FP64 messenger's
    stage lengths and its map to 1e-6."""
    kw = {"discs": 40} if kind == "scan" else {}
    p, d = problem(osht, kind, nside, seed, **kw)
    _, m64, s64, t64 = gpu_solve(torch_cuda, p, d, eps_final=1e-6, precision=0)
    _, m32, s32, t32 = gpu_solve(torch_cuda, p, d, eps_final=1e-6, precision=1)
    assert s64["converged"] == 1 and s32["converged"] == 1
    assert np.array_equal(np.bincount(np.asarray(t32["stage"])),
                          np.bincount(np.asarray(t64["stage"])))
    assert np.linalg.norm(m32 - m64) / np.linalg.norm(m64) < 1e-6
