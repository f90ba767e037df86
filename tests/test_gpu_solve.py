"""The dual messenger solve of the CUDA path (through the C ABI) against the
oracle: dense fixed points, the uniform-noise closed form, the oracle's own
iteration trace, and the diagnostics of App. C."""
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
    elif kind == "scan":
        p = inputs.scan_problem(nside, seed=seed, **kw)
    else:
        p = inputs.uniform_problem(nside, seed=seed, **kw)
    d = p.data(osht.alm2map(p.alm_true, p.nside, p.lmax))
    return p, d


def gpu_solve(torch, p, d, tuning=None, **opts):
    from paper_1702_08852_gb300 import wf
    nv = torch.from_numpy(p.noise_var).cuda()
    mk = torch.from_numpy(p.mask.astype(np.uint8)).cuda()
    with wf.Plan(p.nside, p.lmax, p.cl, nv, mk, **opts) as plan:
        if tuning:
            plan.set_tuning(**tuning)
        alm, mp, st = plan.solve(torch.from_numpy(d).cuda())
        tr = plan.trace()
        return alm.cpu().numpy(), mp.cpu().numpy(), st, tr


def rel_alm(osht, a, b, lmax):
    return osht.alm_norm(a - b, lmax) / osht.alm_norm(b, lmax)


@pytest.mark.parametrize("nside,kind,seed", [(4, "lognormal", 1), (8, "lognormal", 2),
                                             (8, "scan", 3)])
def test_fp64_solve_matches_dense_fixed_point(torch_cuda, osht, odm, nside, kind, seed):
    torch = torch_cuda
    kw = {"discs": 5, "disc_radius_deg": 10.0} if kind == "scan" else {}
    p, d = problem(osht, kind, nside, seed, **kw)
    alm, mp, st, _ = gpu_solve(torch, p, d, eps_final=1e-13)
    assert st["converged"] == 1
    ref = odm.dm_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 0.0)
    assert rel_alm(osht, alm, ref, p.lmax) < 1e-10
    sref = osht.alm2map(ref, p.nside, p.lmax)
    assert np.linalg.norm(mp - sref) / np.linalg.norm(sref) < 1e-10


def test_fp64_solve_nside32_workload(torch_cuda, osht, odm):
    """Nside 32, lmax 64, lognormal noise, |b| < 15 deg band + 20 discs of
    3 deg: the small full-size workload, against the dense fixed point."""
    torch = torch_cuda
    p, d = problem(osht, "lognormal", 32, 1000)
    alm, mp, st, _ = gpu_solve(torch, p, d, eps_final=1e-12, stop_rule=1)
    assert st["converged"] == 1
    Y = osht.ymatrix(p.nside, p.lmax)
    ref = odm.dm_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 0.0, Y=Y)
    sref = Y @ osht.alm_to_real(ref, p.lmax)
    assert np.linalg.norm(mp - sref) / np.linalg.norm(sref) < 1e-10


def test_error_stop_rule_1e6(torch_cuda, osht, odm):
    """The default last-stage stop (error estimate < 1e-6) gives a map within
    a few 1e-6 of the converged solution."""
    torch = torch_cuda
    p, d = problem(osht, "lognormal", 16, 7)
    alm, mp, st, _ = gpu_solve(torch, p, d, stop_rule=1)
    ref = odm.dm_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 0.0)
    sref = osht.alm2map(ref, p.nside, p.lmax)
    assert np.linalg.norm(mp - sref) / np.linalg.norm(sref) < 3e-6


@pytest.mark.parametrize("nside", [8, 64])
def test_uniform_noise_closed_form(torch_cuda, osht, nside):
    torch = torch_cuda
    p, d = problem(osht, "uniform", nside, 4)
    alm, mp, st, tr = gpu_solve(torch, p, d, eps_final=1e-12)
    om = 4 * np.pi / (12 * nside * nside)
    from paper_1702_08852_gb300 import inputs
    ls, _ = inputs.lm_of_slots(p.lmax)
    s2 = p.noise_var[0]
    want = (p.cl / (p.cl + s2 * om))[ls] * osht.map2alm(d, nside, p.lmax)
    assert rel_alm(osht, alm, want, p.lmax) < 1e-12
    assert st["iterations"] <= 2 * st["stages"] + 1


def test_trace_follows_the_oracle(torch_cuda, osht, odm):
    """Same stage schedule and per-iteration Cauchy ratios as the oracle's
    Algorithm 2 (up to rounding, over the first stages)."""
    torch = torch_cuda
    p, d = problem(osht, "lognormal", 8, 12)
    otr = []
    odm.dual_messenger(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d,
                       eps_final=1e-8, stop="error", trace=otr)
    _, _, st, tr = gpu_solve(torch, p, d, eps_final=1e-8, stop_rule=1)
    ost = np.array([t[0] for t in otr])
    oc = np.array([t[3] for t in otr])
    n = min(len(oc), len(tr["cauchy"]), 200)
    assert np.array_equal(tr["stage"][:n], ost[:n])
    assert np.allclose(tr["xi"][:n], [t[1] for t in otr[:n]], rtol=1e-14)
    assert np.allclose(tr["cauchy"][:n], oc[:n], rtol=1e-8, atol=1e-14)
    assert abs(st["iterations"] - len(otr)) <= max(3, len(otr) // 100)


def test_residual_diagnostics(torch_cuda, osht, odm):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    p, d = problem(osht, "lognormal", 8, 21)
    T = odm.MatrixTransforms(p.nside, p.lmax)
    xw = odm.wf_exact_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, Y=T.Y)
    xd = odm.dm_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 0.0, Y=T.Y)
    nv = torch.from_numpy(p.noise_var).cuda()
    mk = torch.from_numpy(p.mask.astype(np.uint8)).cuda()
    dd = torch.from_numpy(d).cuda()
    with wf.Plan(p.nside, p.lmax, p.cl, nv, mk) as plan:
        for x in (xw, xd):
            r = plan.residual(dd, torch.from_numpy(x).cuda())
            assert r["rel_res_wf"] == pytest.approx(
                odm.wf_residual(x, p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, T),
                rel=1e-8, abs=1e-13)
            assert r["chi2"] == pytest.approx(
                odm.chi2(x, p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, T), rel=1e-11)
            assert r["rel_res_fp"] == pytest.approx(
                odm.fixed_point_residual(x, p.nside, p.lmax, p.cl, p.noise_var, p.mask,
                                         d, T), rel=1e-6, abs=1e-13)


def test_host_entry_point_equals_device(torch_cuda, osht):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    p, d = problem(osht, "lognormal", 8, 30)
    nv = torch.from_numpy(p.noise_var).cuda()
    mk = torch.from_numpy(p.mask.astype(np.uint8)).cuda()
    with wf.Plan(p.nside, p.lmax, p.cl, nv, mk) as plan:
        a1, m1, _ = plan.solve(torch.from_numpy(d).cuda())
        a2, m2, _ = plan.solve_host(d)
        assert np.array_equal(a1.cpu().numpy(), a2)
        assert np.array_equal(m1.cpu().numpy(), m2)


def test_cauchy_rule_matches_oracle_and_mixed(torch_cuda, osht, odm):
    """The paper's criterion (Cauchy ratio < eps in the last stage): FP64
    stops at the oracle's iteration and result; the mixed path stops with a
    Cauchy ratio below eps as well."""
    torch = torch_cuda
    p, d = problem(osht, "lognormal", 8, 41)
    otr = []
    xo, info = odm.dual_messenger(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d,
                                  eps_final=1e-6, stop="cauchy", trace=otr)
    alm, mp, st, tr = gpu_solve(torch, p, d, eps_final=1e-6)
    assert abs(st["iterations"] - info["iterations"]) <= 2
    assert rel_alm(osht, alm, xo, p.lmax) < 1e-8
    alm2, mp2, st2, tr2 = gpu_solve(torch, p, d, eps_final=1e-6, precision=1)
    assert st2["converged"] == 1 and tr2["cauchy"][-1] < 1e-6
    # the mixed path reproduces the FP64 result under the same rule
    assert np.linalg.norm(mp2 - mp) / np.linalg.norm(mp) < 1e-6
    assert st2["iterations"] == st["iterations"]


def test_deterministic(torch_cuda, osht):
    torch = torch_cuda
    p, d = problem(osht, "scan", 16, 5, discs=10)
    a1, _, s1, _ = gpu_solve(torch, p, d)
    a2, _, s2, _ = gpu_solve(torch, p, d)
    assert np.array_equal(a1, a2) and s1["iterations"] == s2["iterations"]


def test_plan_rejects_bad_noise(torch_cuda):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    nside, lmax = 4, 8
    nv = torch.ones(12 * nside * nside, dtype=torch.float64, device="cuda")
    nv[3] = -1.0
    with pytest.raises(wf.WFError) as e:
        wf.Plan(nside, lmax, np.ones(lmax + 1), nv)
    assert e.value.status == wf.WF_ERR_ARG
    mk = torch.ones(12 * nside * nside, dtype=torch.uint8, device="cuda")
    with pytest.raises(wf.WFError):
        wf.Plan(nside, lmax, np.ones(lmax + 1), torch.ones_like(nv), mk)
    nv[3] = 1.0
    mk[:] = 0
    mk[3] = 1
    nv[3] = float("nan")   # masked: ignored
    wf.Plan(nside, lmax, np.ones(lmax + 1), nv, mk).close()


@pytest.mark.parametrize("nside,kind,seed,anchor", [(16, "lognormal", 8, 1),
                                                    (16, "lognormal", 8, 0),
                                                    (32, "lognormal", 1000, 1),
                                                    (32, "scan", 9, 1)])
def test_mixed_precision_reaches_fp64_fixed_point(torch_cuda, osht, odm, nside, kind, seed,
                                                  anchor):
    """FP32 transforms for the cooling stages, anchored later stages (anchor
    steps in double-float or plain FP64): the result matches the FP64 fixed
    point (dense solve) to 1e-6 relative L2."""
    torch = torch_cuda
    kw = {"discs": 40} if kind == "scan" else {}
    p, d = problem(osht, kind, nside, seed, **kw)
    alm, mp, st, tr = gpu_solve(torch, p, d, precision=1, eps_final=1e-7, stop_rule=1,
                                anchor=anchor)
    assert st["converged"] == 1
    assert st["refinements"] >= 1
    Y = osht.ymatrix(p.nside, p.lmax)
    ref = odm.dm_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 0.0, Y=Y)
    sref = Y @ osht.alm_to_real(ref, p.lmax)
    err = np.linalg.norm(mp - sref) / np.linalg.norm(sref)
    assert err < 1e-6, (err, st)
    assert st["fp_residual"] < 1e-6


@pytest.mark.parametrize("ana_np,ana_queue,packed,gacc", [(4, 1, 0, 0), (8, 1, 0, 0),
                                                          (16, 0, 0, 0), (2, 0, 0, 0),
                                                          (8, 0, 1, 0), (4, 0, 1, 0),
                                                          (6, 0, 1, 0), (4, 0, 1, 1),
                                                          (8, 0, 1, 2), (4, 0, 1, 2),
                                                          (8, 0, 1, 3)])
def test_mixed_precision_variants_reach_fp64_fixed_point(torch_cuda, osht, odm, ana_np,
                                                         ana_queue, packed, gacc):
    """The same check with the FP32 analysis forced to each launch variant
    (the queue-scheduled one included: its combine kernel carries the filter,
    the anchored-stage source and the Cauchy partial sums)."""
    torch = torch_cuda
    p, d = problem(osht, "lognormal", 16, 8)
    tuning = {"ana_np": (4, ana_np), "ana_queue": ana_queue, "ana_packed": packed,
              "ana_global_acc": gacc}
    if packed:
        tuning.update(syn_np=(2, 2), syn_packed=1)
    alm, mp, st, tr = gpu_solve(torch, p, d, tuning=tuning,
                                precision=1, eps_final=1e-7, stop_rule=1)
    assert st["converged"] == 1
    Y = osht.ymatrix(p.nside, p.lmax)
    ref = odm.dm_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 0.0, Y=Y)
    sref = Y @ osht.alm_to_real(ref, p.lmax)
    assert np.linalg.norm(mp - sref) / np.linalg.norm(sref) < 1e-6


@pytest.mark.parametrize("nside,kind,seed", [(32, "scan", 9), (32, "lognormal", 1000)])
def test_mixed_stage_lengths_match_fp64(torch_cuda, osht, nside, kind, seed):
    """Algorithm 2 carries the messenger t across each cooling step; the mixed
    solver's anchored stages do the same, so stage by stage they take the
    plain FP64 solve's number of iterations (restarting a stage from G(x)
    instead would converge to the same fixed point in more iterations)."""
    torch = torch_cuda
    kw = {"discs": 40} if kind == "scan" else {}
    p, d = problem(osht, kind, nside, seed, **kw)
    _, _, st64, tr64 = gpu_solve(torch, p, d, precision=0)
    _, _, st32, tr32 = gpu_solve(torch, p, d, precision=1)
    assert st64["converged"] == 1 and st32["converged"] == 1
    assert st32["refinements"] >= 1  # anchored stages were run
    n64 = np.bincount(np.asarray(tr64["stage"]))
    n32 = np.bincount(np.asarray(tr32["stage"]))
    assert np.array_equal(n32, n64), (n32, n64)


@pytest.mark.parametrize("nside,lsig", [(128, 256), (256, 128)])
def test_mixed_matches_fp64_solve_at_scale(torch_cuda, osht, nside, lsig):
    """The scan-noise workload (hits 1-100, 25 % mask: galactic band and 500
    discs of 0.5 deg) at Nside 128 and 256 (lmax 2 Nside; the signal of the
    data map band-limited to lsig so that the oracle synthesises it in
    seconds): under the paper's Cauchy rule the mixed path takes the FP64
    solve's stage lengths and its map is within 1e-6 relative L2 of the FP64
    map."""
    torch = torch_cuda
    from paper_1702_08852_gb300 import inputs
    p = inputs.scan_problem(nside, seed=11, mask_fraction=0.25, discs=500,
                            disc_radius_deg=0.5)
    ls, _ = inputs.lm_of_slots(p.lmax)
    a = p.alm_true[ls <= lsig] if lsig < p.lmax else p.alm_true
    d = p.data(osht.alm2map(a, p.nside, min(lsig, p.lmax)))
    _, m64, st64, tr64 = gpu_solve(torch, p, d, precision=0, eps_final=1e-6)
    _, m32, st32, tr32 = gpu_solve(torch, p, d, precision=1, eps_final=1e-6)
    assert st64["converged"] == 1 and st32["converged"] == 1
    n64 = np.bincount(np.asarray(tr64["stage"]))
    n32 = np.bincount(np.asarray(tr32["stage"]))
    assert np.array_equal(n32, n64), (n32, n64)
    err = np.linalg.norm(m32 - m64) / np.linalg.norm(m64)
    assert err < 1e-6, err


def test_set_cl_equals_a_plan_made_with_it(torch_cuda, osht):
    """wf_set_cl refreshes every copy of C_l the solver reads (the FP64 one
    and the FP32 one of the mixed path's FP32 stages): a plan made with C_l
    and then given 1.7 C_l solves exactly as a plan made with 1.7 C_l."""
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    p, d = problem(osht, "lognormal", 16, 12)
    cl2 = 1.7 * p.cl
    nv = torch.from_numpy(p.noise_var).cuda()
    mk = torch.from_numpy(p.mask.astype(np.uint8)).cuda()
    dt = torch.from_numpy(d).cuda()
    out = []
    for cl_make, cl_set in ((p.cl, cl2), (cl2, None)):
        with wf.Plan(p.nside, p.lmax, cl_make, nv, mk, precision=1, eps_final=1e-7) as plan:
            if cl_set is not None:
                plan.set_cl(cl_set)
            alm, _, st = plan.solve(dt)
            out.append((alm.cpu().numpy(), st["iterations"]))
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])
