"""Learned warm start: training and use of the network of include/wf.h
(wf_net_*).  Every numerical step runs in the library's kernels; this module
only orchestrates (data generation with the plain solver, epochs, the
warm-or-cold decision).

The net maps (d, log sigma^2, mask) to (t0, a0).  A warm solve starts
Algorithm 2 from (a0, t0) with a cooling start mu0 = mu0_over_alpha * alpha
instead of the cold start (s = 0, t = d, mu0 Omega = beta max C_l).  It is
used only when it helps on the problem at hand: if the Wiener-filter residual
||A x - y|| / ||y|| (App. C) of a0 is not below that of the zero start
(which is 1), the cold start is used instead.
"""
import numpy as np

from . import wf


def init_params(channels, kernel, hidden, seed=0):
    """He-style random initial weights (numpy RNG), biases 0; the last conv
    layer starts at 0 so the untrained net returns the masked data."""
    rng = np.random.default_rng(seed)
    H, K, Hm = channels, kernel, hidden
    parts = [np.sqrt(2.0 / (3 * K)) * rng.standard_normal(H * 3 * K), np.zeros(H),
             np.sqrt(2.0 / (H * K)) * rng.standard_normal(H * H * K), np.zeros(H),
             np.zeros(H * K), np.zeros(1),
             np.sqrt(2.0 / 4) * rng.standard_normal(Hm * 4), np.zeros(Hm),
             np.sqrt(2.0 / Hm) * rng.standard_normal(Hm * Hm), np.zeros(Hm),
             np.sqrt(1.0 / Hm) * rng.standard_normal(Hm), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


def train(net, samples, epochs=20, lr=3e-3, seed=0, plans=None, log=None):
    """samples: list of (plan, d, target_alm); the net is trained on each
    sample with that sample's plan (noise, mask, spectrum).  Plans must share
    the geometry of the net's plan; the net reads the plan it was created
    with, so each sample's noise/mask/spectrum is loaded into it first."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(samples))
        tot = 0.0
        for i in order:
            nv, mk, cl, d, target = samples[i]
            net.plan.set_noise(nv, mk)
            net.plan.set_cl(cl)
            loss, _ = net.loss_grad(d, target)
            net.adam_step(lr)
            tot += loss
        hist.append(tot / len(samples))
        if log:
            log(ep, hist[-1])
    return hist


def warm_solve(net, plan, d, mu0_over_alpha=30.0):
    """Solve with the net's warm start when it beats the zero start (see the
    module docstring).  ``plan`` must be the net's plan geometry with the
    problem's noise/mask/spectrum and its cooling start set to
    mu0_over_alpha * alpha.  Returns (alm, map, stats, used_warm, residual)."""
    t0, a0 = net.forward(d)
    res = plan.residual(d, a0)["rel_res_wf"]
    if not (res < 1.0):
        alm, mp, st = plan.solve(d)
        return alm, mp, st, False, res
    alm, mp, st = plan.solve(d, init_alm=a0, init_map=t0)
    return alm, mp, st, True, res
