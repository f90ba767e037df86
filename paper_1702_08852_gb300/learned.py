"""Learned warm start: training and use of the network of include/wf.h
(wf_net_*).  Every numerical step runs in the library's kernels; this module
only orchestrates (data generation with the plain solver, epochs, the
warm-or-cold decision).

The net maps (d, log sigma^2, mask) to (t0, a0).  A warm solve starts
Algorithm 2 from (a0, t0) with a cooling start mu0 = mu0_over_alpha * alpha
instead of the cold start (s = 0, t = d, mu0 Omega = beta max C_l), i.e. it
skips the stages above mu0.  The plain method decides on the warm start: it is
used only if its Wiener-filter residual ||A x - y|| / ||y|| (App. C) is
below both the zero start's (1) and the tolerance of the stage it enters,
eps_k = min(eps_cap, eps_final mu0 / alpha); the cold stages would hand that
stage an iterate within its tolerance, and a start farther away costs more
late-stage iterations than the skipped early stages save.  Otherwise the
cold start is used.
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


def entry_tolerance(plan, mu0_over_alpha):
    o = plan.opts
    return min(o.eps_cap, o.eps_final * max(1.0, mu0_over_alpha))


def warm_solve(net, plan, d, cold_plan, mu0_over_alpha=30.0):
    """Solve with the net's warm start when the plain method accepts it (see
    the module docstring).  ``plan`` is the net's plan (the problem's noise,
    mask, spectrum) with its cooling start set to mu0_over_alpha * alpha;
    ``cold_plan`` (required) is a plan of the same problem with the plain
    method's cooling start, which runs the cold start when the warm one is
    rejected.  Returns (alm, map, stats, used_warm, residual)."""
    if cold_plan is None:
        raise ValueError("warm_solve: cold_plan is required (the plain method's "
                         "cold start is the fallback)")
    t0, a0 = net.forward(d)
    res = plan.residual(d, a0)["rel_res_wf"]
    if res < min(1.0, entry_tolerance(plan, mu0_over_alpha)):
        alm, mp, st = plan.solve(d, init_alm=a0, init_map=t0)
        return alm, mp, st, True, res
    alm, mp, st = cold_plan.solve(d)
    return alm, mp, st, False, res
