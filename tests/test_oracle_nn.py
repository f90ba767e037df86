"""The FP64 reference of the warm-start network: its hand-written gradient
against central finite differences."""
import numpy as np
import pytest


def setup(osht, nside=4, H=3, K=3, Hm=5, seed=0):
    from oracle import nn
    from paper_1702_08852_gb300 import inputs
    p = inputs.lognormal_problem(nside, seed=seed, band_deg=20.0, discs=2)
    d = p.data(osht.alm2map(p.alm_true, p.nside, p.lmax))
    rng = np.random.default_rng(seed + 1)
    _, n = nn.layout(H, K, Hm)
    theta = 0.3 * rng.standard_normal(n)
    target = p.alm_true * 0.8
    return p, d, theta, target, (H, K, Hm)


def test_gradient_matches_finite_differences(osht):
    from oracle import nn
    p, d, theta, target, (H, K, Hm) = setup(osht)
    loss, g = nn.loss_grad(theta, H, K, Hm, p.nside, p.lmax, p.cl, p.noise_var, p.mask,
                           d, target)
    assert np.isfinite(loss) and loss > 0
    rng = np.random.default_rng(5)
    idx = rng.choice(len(theta), 25, replace=False)
    for i in idx:
        e = np.zeros_like(theta)
        h = 1e-6
        e[i] = h
        lp, _ = nn.loss_grad(theta + e, H, K, Hm, p.nside, p.lmax, p.cl, p.noise_var,
                             p.mask, d, target)
        lm, _ = nn.loss_grad(theta - e, H, K, Hm, p.nside, p.lmax, p.cl, p.noise_var,
                             p.mask, d, target)
        fd = (lp - lm) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9)


def test_zero_network_is_the_masked_data_filtered(osht):
    """With all weights zero, t0 is the masked data and the gain is 1/2."""
    from oracle import nn
    p, d, theta, target, (H, K, Hm) = setup(osht)
    st = nn.forward(np.zeros_like(theta), H, K, Hm, p.nside, p.lmax, p.cl, p.noise_var,
                    p.mask, d)
    assert np.allclose(st["t0"], np.where(p.mask, 0.0, d))
    assert np.allclose(st["q"], 0.5)
    assert np.allclose(st["a0"], 0.5 * osht.map2alm(np.where(p.mask, 0.0, d), p.nside, p.lmax))
