"""Batched solves (many maps of uneven Nside, noise and mask together) and
the launch-variant autotuner, through the C ABI."""
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


def make_problems(osht, specs):
    from paper_1702_08852_gb300 import inputs
    out = []
    for kind, ns, seed in specs:
        if kind == "lognormal":
            p = inputs.lognormal_problem(ns, seed=seed)
        else:
            p = inputs.scan_problem(ns, seed=seed, discs=10, amplitude=1.5)
        out.append((p, p.data(osht.alm2map(p.alm_true, p.nside, p.lmax))))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_one_by_one(torch_cuda, osht, precision):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    probs = make_problems(osht, [("lognormal", 8, 1), ("scan", 16, 2), ("lognormal", 16, 3),
                                 ("scan", 32, 4), ("lognormal", 4, 5), ("scan", 8, 6)])
    plans, ds, single = [], [], []
    for p, d in probs:
        nv = torch.from_numpy(p.noise_var).cuda()
        mk = torch.from_numpy(p.mask.astype(np.uint8)).cuda()
        plan = wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=precision)
        dd = torch.from_numpy(d).cuda()
        a, _, st = plan.solve(dd, want_map=False)
        single.append((a.cpu().numpy(), st["iterations"]))
        plans.append(plan)
        ds.append(dd)
    alms, maps, stats, ms = wf.wf_solve_batch(plans, ds, want_map=True)
    assert ms > 0
    for (a1, it1), a2, m2, st, plan in zip(single, alms, maps, stats, plans):
        assert np.array_equal(a1, a2.cpu().numpy())
        assert st["iterations"] == it1 and st["converged"] == 1
        assert np.array_equal(plan.alm2map(a2).cpu().numpy(), m2.cpu().numpy())
    for plan in plans:
        plan.close()


def test_batch_with_more_maps_than_host_threads(torch_cuda, osht):
    """More maps than the pool has threads (one per core): the queue hands
    each thread several maps, largest first; every result equals its
    one-by-one solve."""
    import os
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    n = (os.cpu_count() or 16) + 5
    specs = [("lognormal" if i % 2 else "scan", 8, 100 + i) for i in range(n)]
    probs = make_problems(osht, specs)
    plans, ds, single = [], [], []
    for p, d in probs:
        nv = torch.from_numpy(p.noise_var).cuda()
        mk = torch.from_numpy(p.mask.astype(np.uint8)).cuda()
        plan = wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=1)
        dd = torch.from_numpy(d).cuda()
        a, _, _ = plan.solve(dd, want_map=False)
        single.append(a.cpu().numpy())
        plans.append(plan)
        ds.append(dd)
    alms, _, stats, _ = wf.wf_solve_batch(plans, ds)
    for a1, a2, st in zip(single, alms, stats):
        assert np.array_equal(a1, a2.cpu().numpy()) and st["converged"] == 1
    for plan in plans:
        plan.close()


def test_batch_rejects_duplicates_and_missing_noise(torch_cuda):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    nv = torch.ones(12 * 16, dtype=torch.float64, device="cuda")
    d = torch.zeros(12 * 16, dtype=torch.float64, device="cuda")
    p1 = wf.Plan(4, 8, np.ones(9), nv)
    p2 = wf.Plan(4, 8, np.ones(9))
    with pytest.raises(wf.WFError):
        wf.wf_solve_batch([p1, p1], [d, d])
    with pytest.raises(wf.WFError):
        wf.wf_solve_batch([p1, p2], [d, d])
    p1.close()
    p2.close()


def test_autotuned_plan_reaches_the_same_fixed_point(torch_cuda, osht, odm):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf
    (p, d), = make_problems(osht, [("lognormal", 16, 11)])
    nv = torch.from_numpy(p.noise_var).cuda()
    mk = torch.from_numpy(p.mask.astype(np.uint8)).cuda()
    ref = odm.dm_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 0.0)
    for prec, tol in ((0, 1e-10), (1, 1e-6)):
        with wf.Plan(p.nside, p.lmax, p.cl, nv, mk, precision=prec, autotune=1,
                     eps_final=1e-12 if prec == 0 else 1e-7, stop_rule=1) as plan:
            a, _, st = plan.solve(torch.from_numpy(d).cuda(), want_map=False)
        a = a.cpu().numpy()
        assert osht.alm_norm(a - ref, p.lmax) / osht.alm_norm(ref, p.lmax) < tol
