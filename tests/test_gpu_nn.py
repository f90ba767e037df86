"""The learned warm start's kernels (forward, loss, backward) against the
FP64 oracle network, training, and warm-started solves."""
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


def problem(osht, nside, seed):
    from paper_1702_08852_gb300 import inputs
    p = inputs.lognormal_problem(nside, seed=seed, band_deg=20.0, discs=3)
    return p, p.data(osht.alm2map(p.alm_true, p.nside, p.lmax))


@pytest.mark.parametrize("nside,H,K,Hm", [(4, 3, 3, 5), (8, 8, 5, 16)])
def test_loss_and_gradient_match_oracle(torch_cuda, osht, nside, H, K, Hm):
    torch = torch_cuda
    from oracle import nn as onn
    from paper_1702_08852_gb300 import wf
    p, d = problem(osht, nside, 3)
    rng = np.random.default_rng(4)
    _, n = onn.layout(H, K, Hm)
    theta = (0.3 * rng.standard_normal(n)).astype(np.float32)
    target = (0.8 * p.alm_true).astype(np.complex128)
    nv = torch.from_numpy(p.noise_var).cuda()
    mk = torch.from_numpy(p.mask.astype(np.uint8)).cuda()
    with wf.Plan(p.nside, p.lmax, p.cl, nv, mk) as plan:
        net = wf.Net(plan, H, K, Hm, bf16=False)
        assert net.nparams == n
        net.set_params(theta)
        loss, g = net.loss_grad(torch.from_numpy(d).cuda(), torch.from_numpy(target).cuda(),
                                want_grad=True)
        t0, a0 = net.forward(torch.from_numpy(d).cuda())
        net.close()
    ref_loss, ref_g = onn.loss_grad(theta.astype(np.float64), H, K, Hm, p.nside, p.lmax, p.cl,
                                    p.noise_var, p.mask, d, target)
    st = onn.forward(theta.astype(np.float64), H, K, Hm, p.nside, p.lmax, p.cl, p.noise_var,
                     p.mask, d)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    assert np.linalg.norm(g - ref_g) <= 1e-3 * np.linalg.norm(ref_g)
    lay, _ = onn.layout(H, K, Hm)
    for name, (o, s) in lay.items():
        sl = slice(o, o + int(np.prod(s)))
        assert np.linalg.norm(g[sl] - ref_g[sl]) <= 2e-3 * np.linalg.norm(ref_g[sl]) + 1e-7, name
    assert np.max(np.abs(t0.cpu().numpy() - st["t0"])) <= 1e-5 * np.max(np.abs(st["t0"]))
    assert np.max(np.abs(a0.cpu().numpy() - st["a0"])) <= 1e-4 * np.max(np.abs(st["a0"]))


def test_bf16_weights_change_little(torch_cuda, osht):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf, learned
    p, d = problem(osht, 8, 5)
    nv = torch.from_numpy(p.noise_var).cuda()
    mk = torch.from_numpy(p.mask.astype(np.uint8)).cuda()
    theta = learned.init_params(8, 5, 16, seed=1)
    theta[-1] = 0.3
    dd = torch.from_numpy(d).cuda()
    tgt = torch.from_numpy(p.alm_true).cuda()
    with wf.Plan(p.nside, p.lmax, p.cl, nv, mk) as plan:
        out = []
        for bf in (False, True):
            net = wf.Net(plan, 8, 5, 16, bf16=bf)
            net.set_params(theta)
            out.append(net.loss_grad(dd, tgt)[0])
            net.close()
    assert out[1] == pytest.approx(out[0], rel=2e-2)


def test_training_lowers_the_loss_and_warm_solve_is_exact(torch_cuda, osht, odm):
    torch = torch_cuda
    from paper_1702_08852_gb300 import wf, learned
    samples = []
    plans = []
    for seed in range(6):
        p, d = problem(osht, 8, 100 + seed)
        nv = torch.from_numpy(p.noise_var).cuda()
        mk = torch.from_numpy(p.mask.astype(np.uint8)).cuda()
        with wf.Plan(p.nside, p.lmax, p.cl, nv, mk, eps_final=1e-12, stop_rule=1) as sp:
            a, _, _ = sp.solve(torch.from_numpy(d).cuda(), want_map=False)
        samples.append((nv, mk, p.cl, torch.from_numpy(d).cuda(), a))
        plans.append(p)
    p0 = plans[0]
    with wf.Plan(p0.nside, p0.lmax, p0.cl, samples[0][0], samples[0][1]) as plan:
        net = wf.Net(plan, 8, 5, 16)
        net.set_params(learned.init_params(8, 5, 16, seed=2))
        hist = learned.train(net, samples, epochs=15, lr=3e-3)
        assert hist[-1] < 0.8 * hist[0]
        # warm solve of a held-out map reaches the same fixed point
        p, d = problem(osht, 8, 999)
        nv = torch.from_numpy(p.noise_var).cuda()
        mk = torch.from_numpy(p.mask.astype(np.uint8)).cuda()
        plan.set_noise(nv, mk)
        plan.set_cl(p.cl)
        alpha = float(np.min(p.noise_var[~p.mask]))
        with wf.Plan(p.nside, p.lmax, p.cl, nv, mk, eps_final=1e-12, stop_rule=1,
                     mu0=30.0 * alpha) as wp, \
                wf.Plan(p.nside, p.lmax, p.cl, nv, mk, eps_final=1e-12, stop_rule=1) as cp:
            wnet = wf.Net(wp, 8, 5, 16)
            wnet.set_params(net.get_params())
            alm, mp, st, used, res = learned.warm_solve(wnet, wp, torch.from_numpy(d).cuda(),
                                                        cold_plan=cp)
            # the acceptance rule: warm only when within the entry stage's tolerance
            assert used == (res < learned.entry_tolerance(wp, 30.0))
            wnet.close()
        net.close()
    ref = odm.dm_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 0.0)
    a = alm.cpu().numpy()
    assert st["converged"] == 1
    assert osht.alm_norm(a - ref, p.lmax) / osht.alm_norm(ref, p.lmax) < 1e-9
