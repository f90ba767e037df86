"""Pins for the oracle's dual messenger (Algorithm 2) and the solves it is
checked against: dense fixed points, the exact Wiener filter (Eq. 2, App. C)
and PCG, the uniform-noise closed form, the alpha / mu limits of Eq. (13)
and the behaviour of the cooling schedule."""
import numpy as np
import pytest

from paper_1702_08852_gb300 import inputs


def make(osht, kind, nside, seed, **kw):
    if kind == "lognormal":
        p = inputs.lognormal_problem(nside, seed=seed, **kw)
    elif kind == "scan":
        p = inputs.scan_problem(nside, seed=seed, discs=5, disc_radius_deg=10.0, **kw)
    else:
        p = inputs.uniform_problem(nside, seed=seed, **kw)
    d = p.data(osht.alm2map(p.alm_true, p.nside, p.lmax))
    return p, d


def rel(osht, a, b, lmax):
    return osht.alm_norm(a - b, lmax) / osht.alm_norm(b, lmax)


@pytest.mark.parametrize("nside,kind", [(4, "lognormal"), (8, "lognormal"),
                                        (8, "scan")])
def test_iteration_reaches_dense_fixed_point(osht, odm, nside, kind):
    p, d = make(osht, kind, nside, seed=11 + nside)
    x, info = odm.dual_messenger(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d,
                                 eps_final=1e-14)
    assert info["converged"]
    xd = odm.dm_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 0.0)
    assert rel(osht, x, xd, p.lmax) < 1e-10


@pytest.mark.parametrize("mu_over_alpha", [30.0, 3.0, 0.5])
def test_dense_fixed_point_matches_inner_loop(osht, odm, mu_over_alpha):
    """The closed-form fixed point at a given mu equals the limit of the
    plain inner loop G at that (xi, mu)."""
    p, d = make(osht, "lognormal", 4, seed=5)
    T = odm.MatrixTransforms(p.nside, p.lmax)
    a = odm.alpha_of(p.noise_var, p.mask)
    mu = mu_over_alpha * a
    x = np.zeros(osht.nalm(p.lmax), dtype=complex)
    for _ in range(20000):
        xn = odm.dm_iterate(x, p.nside, p.lmax, p.cl, p.noise_var, p.mask, d,
                            a + mu, mu, T)
        done = osht.alm_norm(xn - x, p.lmax) < 1e-15 * osht.alm_norm(xn, p.lmax)
        x = xn
        if done:
            break
    xd = odm.dm_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, mu)
    assert rel(osht, x, xd, p.lmax) < 1e-11


@pytest.mark.parametrize("nside", [4, 8])
def test_uniform_noise_closed_form(osht, odm, nside):
    """N = sigma^2 1, no mask: the messenger is exact in one step per stage
    (Sect. 2.1, Eq. A4) and the result is s_lm = C_l / (C_l + sigma^2 Omega)
    (Omega Y^T d)_lm."""
    p, d = make(osht, "uniform", nside, seed=2)
    x, info = odm.dual_messenger(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d,
                                 eps_final=1e-12)
    assert info["iterations"] <= 2 * info["stages"]
    om = 4 * np.pi / osht.npix(nside)
    ls, _ = osht.lm_arrays(p.lmax)
    s2 = p.noise_var[0]
    want = (p.cl / (p.cl + s2 * om))[ls] * osht.map2alm(d, nside, p.lmax)
    assert rel(osht, x, want, p.lmax) < 1e-12


def test_exact_wf_three_ways(osht, odm):
    """Eq. (2) solved densely in App. C's symmetric form, densely in the
    C^-1 form on l >= 2, and by PCG with the harmonic-diagonal
    preconditioner (App. C) agree."""
    p, d = make(osht, "lognormal", 4, seed=9)
    lmax = p.lmax
    xa = odm.wf_exact_dense(p.nside, lmax, p.cl, p.noise_var, p.mask, d)
    Y = osht.ymatrix(p.nside, lmax)
    ell = osht.real_ell(lmax)
    keep = ell >= 2
    Yk = Y[:, keep]
    ninv = np.where(p.mask, 0.0, 1.0 / p.noise_var)
    A = np.diag(1.0 / p.cl[ell[keep]]) + Yk.T @ (ninv[:, None] * Yk)
    xk = np.linalg.solve(A, Yk.T @ (ninv * d))
    xr = np.zeros(Y.shape[1])
    xr[keep] = xk
    xb = osht.real_to_alm(xr, lmax)
    assert rel(osht, xa, xb, lmax) < 1e-10
    xp, info = odm.pcg_wf(p.nside, lmax, p.cl, p.noise_var, p.mask, d, tol=1e-13)
    assert info["rel_residual"] < 1e-13
    assert rel(osht, xp, xa, lmax) < 1e-10
    T = odm.MatrixTransforms(p.nside, lmax, Y)
    assert odm.wf_residual(xa, p.nside, lmax, p.cl, p.noise_var, p.mask, d, T) < 1e-13


@pytest.mark.parametrize("nside", [4, 8])
def test_gap_to_exact_wf_is_quadrature(osht, odm, nside):
    """The messenger's fixed point is the exact Wiener filter only when the
    basis change is orthogonal (Sect. 2.1).  On HEALPix the gap is of the
    order of the quadrature error of Omega Y^T Y; it is reported, and it
    vanishes when Y is replaced by an orthonormalised copy."""
    p, d = make(osht, "lognormal", nside, seed=21)
    lmax = p.lmax
    xd = odm.dm_fixed_point_dense(p.nside, lmax, p.cl, p.noise_var, p.mask, d, 0.0)
    xw = odm.wf_exact_dense(p.nside, lmax, p.cl, p.noise_var, p.mask, d)
    gap = rel(osht, xd, xw, lmax)
    assert 1e-4 < gap < 0.2
    # orthonormalise Y (keeps the column space): Omega Q^T Q = 1 exactly
    Y = osht.ymatrix(p.nside, lmax)
    om = 4 * np.pi / osht.npix(p.nside)
    Q, R = np.linalg.qr(Y * np.sqrt(om))
    R = R * np.sign(np.diag(R))[:, None]
    Q = Y @ np.linalg.inv(R)          # Omega Q^T Q = 1
    assert np.max(np.abs(om * Q.T @ Q - np.eye(Q.shape[1]))) < 1e-10
    # with a diagonal prior in the Q basis both solves coincide
    xq = odm.dm_fixed_point_dense(p.nside, lmax, p.cl, p.noise_var, p.mask, d, 0.0, Y=Q)
    xwq = odm.wf_exact_dense(p.nside, lmax, p.cl, p.noise_var, p.mask, d, Y=Q)
    assert rel(osht, xq, xwq, lmax) < 1e-10


def test_limits_of_the_hybrid_equations(odm):
    """Eq. (13)-(15): with alpha = 0 the pixel and harmonic steps are the
    pure dual messenger equations (9)-(10); with mu = 0 they are the standard
    messenger equations (4)-(5) at lambda = 1."""
    rng = np.random.default_rng(0)
    n = 200
    s2 = rng.uniform(1.0, 5.0, n)
    d, s = rng.standard_normal(n), rng.standard_normal(n)
    mask = np.zeros(n, dtype=bool)
    # alpha = 0, U = mu: (N^-1 + U^-1) t = N^-1 d + U^-1 s
    mu = 0.7
    t = s + odm.pixel_weight(s2, mask, mu, mu) * (d - s)
    assert np.allclose((1 / s2 + 1 / mu) * t, d / s2 + s / mu, rtol=1e-13)
    # mu = 0, xi = alpha, Nbar = N - alpha: (Nbar^-1 + alpha^-1) t = Nbar^-1 d + alpha^-1 s
    alpha = 0.9
    t = s + odm.pixel_weight(s2, mask, alpha, 0.0) * (d - s)
    nb = s2 - alpha
    assert np.allclose((1 / nb + 1 / alpha) * t, d / nb + s / alpha, rtol=1e-12)
    # harmonic step (U^-1 + Sbar^-1) u = U^-1 t  <=>  u = Sbar/(Sbar+U) t
    cl = rng.uniform(0.0, 3.0, 50)
    om = 0.1
    f = odm.filter_ell(cl, mu, mu, om)
    sbar = np.maximum(cl - mu * om, 0.0)
    tt = rng.standard_normal(50)
    u = f * tt
    pos = sbar > 0
    assert np.allclose((1 / (mu * om) + 1 / sbar[pos]) * u[pos], tt[pos] / (mu * om))
    assert np.all(u[~pos] == 0)


def test_cooling_brings_residual_and_chi2_down(osht, odm):
    """End-of-stage iterates approach the solution as xi cools to alpha: the
    Wiener-filter residual (App. C) and chi^2 at the end of each stage do not
    grow from stage to stage (Sect. 4, Figs. 5 and 6)."""
    p, d = make(osht, "lognormal", 8, seed=33)
    T = odm.MatrixTransforms(p.nside, p.lmax)
    res, chi = [], []

    def cb(stage, xi, mu, x):
        res.append(odm.fixed_point_residual(x, p.nside, p.lmax, p.cl, p.noise_var,
                                            p.mask, d, T))
        chi.append(odm.chi2(x, p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, T))

    odm.dual_messenger(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d,
                       eps_final=1e-10, transforms=T, stage_callback=cb)
    assert len(res) > 5
    assert all(b <= a * (1 + 1e-9) for a, b in zip(res, res[1:]))
    assert all(b <= a * (1 + 1e-9) for a, b in zip(chi, chi[1:]))
    assert res[-1] < 1e-9


def test_error_stop_rule_meets_its_tolerance(osht, odm):
    """The last-stage stop on the geometric error estimate delivers the
    requested accuracy (the Cauchy ratio alone does not, Sect. 3)."""
    p, d = make(osht, "lognormal", 8, seed=44)
    T = odm.MatrixTransforms(p.nside, p.lmax)
    xd = odm.dm_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 0.0, Y=T.Y)
    sd = T.synth(xd)
    for tol in (1e-5, 1e-7):
        x, _ = odm.dual_messenger(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d,
                                  eps_final=tol, stop="error", transforms=T)
        err = np.linalg.norm(T.synth(x) - sd) / np.linalg.norm(sd)
        assert err < 3 * tol


def test_pcg_cauchy_rule_of_app_c(osht, odm):
    """App. C's stop rule ||z_{i+1} - z_i|| / ||z_{i+1}|| < eps: the step norm
    it tests is |alpha| ||p|| (z_{i+1} = z_i + alpha p), and the solve it ends
    is within the rule's reach of the exact Wiener filter."""
    p, d = make(osht, "lognormal", 4, seed=19)
    xa = odm.wf_exact_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d)
    x6, i6 = odm.pcg_wf(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, tol=1e-6,
                        stop="cauchy")
    assert i6["cauchy"] < 1e-6
    x12, i12 = odm.pcg_wf(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, tol=1e-12,
                          stop="cauchy")
    assert i12["iterations"] > i6["iterations"]
    assert rel(osht, x12, xa, p.lmax) < 1e-9
    assert rel(osht, x6, xa, p.lmax) < 1e-3
