"""Pins for the oracle's standard messenger (Algorithm 1, Sect. 2.1): the
uniform-noise closed form, dense fixed points at fixed lambda, the error
propagation of Eq. (6), the lambda = 1 fixed point (shared with Algorithm 2's
last stage, and the exact Wiener filter when the basis change is
orthogonal), and the behaviour of the lambda cooling."""
import numpy as np
import pytest

from paper_1702_08852_gb300 import inputs


@pytest.fixture(scope="module")
def omsg():
    from oracle import messenger
    return messenger


def make(osht, kind, nside, seed, **kw):
    if kind == "lognormal":
        p = inputs.lognormal_problem(nside, seed=seed, **kw)
    else:
        p = inputs.uniform_problem(nside, seed=seed, **kw)
    d = p.data(osht.alm2map(p.alm_true, p.nside, p.lmax))
    return p, d


def rel(osht, a, b, lmax):
    return osht.alm_norm(a - b, lmax) / osht.alm_norm(b, lmax)


@pytest.mark.parametrize("nside", [4, 8])
def test_uniform_noise_closed_form(osht, omsg, nside):
    """N = sigma^2 1, no mask: Nbar = 0, so t = d and every stage is exact in
    one step; the lambda = 1 result is s_lm = C_l / (C_l + sigma^2 Omega)
    (Omega Y^T d)_lm."""
    p, d = make(osht, "uniform", nside, seed=2)
    x, info = omsg.standard_messenger(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d,
                                      eps_final=1e-12)
    assert info["converged"] and info["iterations"] <= 2 * info["stages"]
    om = 4 * np.pi / osht.npix(nside)
    ls, _ = osht.lm_arrays(p.lmax)
    want = (p.cl / (p.cl + p.noise_var[0] * om))[ls] * osht.map2alm(d, nside, p.lmax)
    assert rel(osht, x, want, p.lmax) < 1e-12


def inner_step(osht, omsg, p, d, lam, a, T, s_alm):
    """One iteration of Algorithm 1's inner loop from the messenger field
    consistent with s (t = s + w (d - s))."""
    ls, _ = osht.lm_arrays(p.lmax)
    dd = np.where(p.mask, 0.0, d)
    sm = T.synth(s_alm)
    t = sm + omsg.messenger_weight(p.noise_var, p.mask, lam, a) * (dd - sm)
    return omsg.signal_filter(p.cl, lam, a, T.omega)[ls] * (T.omega * T.adjoint(t))


@pytest.mark.parametrize("lam", [30.0, 3.0, 1.0])
def test_dense_fixed_point_matches_inner_loop(osht, odm, omsg, lam):
    p, d = make(osht, "lognormal", 4, seed=5)
    T = odm.MatrixTransforms(p.nside, p.lmax)
    a = odm.alpha_of(p.noise_var, p.mask)
    x = np.zeros(osht.nalm(p.lmax), dtype=complex)
    for _ in range(40000):
        xn = inner_step(osht, omsg, p, d, lam, a, T, x)
        done = osht.alm_norm(xn - x, p.lmax) < 1e-15 * osht.alm_norm(xn, p.lmax)
        x = xn
        if done:
            break
    xd = omsg.messenger_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, lam)
    assert rel(osht, x, xd, p.lmax) < 1e-11


def test_error_propagation_of_eq6(osht, odm, omsg):
    """Eq. (6): the difference of two iterates maps as
    e <- [S (S + lambda T)^-1] [Nbar (Nbar + lambda T)^-1] e, i.e.
    F Omega Y^T (1 - W) Y on the sphere."""
    p, d = make(osht, "lognormal", 4, seed=6)
    T = odm.MatrixTransforms(p.nside, p.lmax)
    a = odm.alpha_of(p.noise_var, p.mask)
    lam = 7.0
    rng = np.random.default_rng(1)
    x1 = inputs.random_alm(rng, p.cl)
    x2 = inputs.random_alm(rng, p.cl)
    e = inner_step(osht, omsg, p, d, lam, a, T, x1) - inner_step(osht, omsg, p, d, lam, a, T, x2)
    Y = T.Y
    ell = osht.real_ell(p.lmax)
    om = T.omega
    S = p.cl[ell]
    nbar = np.where(p.mask, np.inf, p.noise_var - a)
    one_minus_w = np.where(p.mask, 1.0, nbar / (nbar + lam * a))
    Fm = S / (S + lam * a * om)
    want = Fm * (om * (Y.T @ (one_minus_w * (Y @ osht.alm_to_real(x1 - x2, p.lmax)))))
    assert rel(osht, e, osht.real_to_alm(want, p.lmax), p.lmax) < 1e-12


@pytest.mark.parametrize("nside", [4, 8])
def test_last_stage_is_algorithm_2s_fixed_point(osht, odm, omsg, nside):
    """At lambda = 1 the messenger's pixel weight alpha / sigma^2 and filter
    C / (C + alpha Omega) are those of Algorithm 2's last stage (xi = alpha,
    mu = 0): the two fixed points coincide."""
    p, d = make(osht, "lognormal", nside, seed=40 + nside)
    xm = omsg.messenger_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 1.0)
    xd = odm.dm_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 0.0)
    assert rel(osht, xm, xd, p.lmax) < 1e-12


def test_orthogonal_basis_gives_the_wiener_filter(osht, odm, omsg):
    """With an orthogonal basis change (Omega Q^T Q = 1) the lambda = 1 fixed
    point solves Eq. (2) exactly (Sect. 2.1)."""
    p, d = make(osht, "lognormal", 4, seed=23)
    Y = osht.ymatrix(p.nside, p.lmax)
    om = 4 * np.pi / osht.npix(p.nside)
    _, R = np.linalg.qr(Y * np.sqrt(om))
    R = R * np.sign(np.diag(R))[:, None]
    Q = Y @ np.linalg.inv(R)
    xm = omsg.messenger_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 1.0,
                                          Y=Q)
    xw = odm.wf_exact_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, Y=Q)
    assert rel(osht, xm, xw, p.lmax) < 1e-10


@pytest.mark.parametrize("nside", [4, 8])
def test_iteration_reaches_dense_fixed_point(osht, odm, omsg, nside):
    p, d = make(osht, "lognormal", nside, seed=11 + nside)
    x, info = omsg.standard_messenger(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d,
                                      eps_final=1e-14, stop="error")
    assert info["converged"]
    xd = omsg.messenger_fixed_point_dense(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, 1.0)
    assert rel(osht, x, xd, p.lmax) < 1e-10


def test_cooling_brings_residual_and_chi2_down(osht, odm, omsg):
    """End-of-stage iterates approach the solution as lambda cools to 1
    (Sect. 4: chi^2 drops with each change of lambda): the residual of the
    lambda = 1 map does not grow from stage to stage, nor does chi^2 beyond
    1e-5 of itself (on HEALPix the lambda = 1 fixed point differs from the
    exact chi^2 minimum by the quadrature gap, so its chi^2 may sit a hair
    above that of the last iterate before it); the tolerances follow the
    three steps."""
    p, d = make(osht, "lognormal", 8, seed=31)
    T = odm.MatrixTransforms(p.nside, p.lmax)
    res, chi, tr = [], [], []

    def cb(stage, lam, x):
        res.append(odm.fixed_point_residual(x, p.nside, p.lmax, p.cl, p.noise_var,
                                            p.mask, d, T))
        chi.append(odm.chi2(x, p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, T))

    omsg.standard_messenger(p.nside, p.lmax, p.cl, p.noise_var, p.mask, d, eps_final=1e-10,
                            transforms=T, trace=tr, stage_callback=cb)
    assert len(res) > 20
    assert all(b <= a * (1 + 1e-9) for a, b in zip(res, res[1:]))
    assert all(b <= a * (1 + 1e-5) for a, b in zip(chi, chi[1:]))
    assert all(b <= a for a, b in zip(chi[:-2], chi[1:-1]))
    assert res[-1] < 1e-9
    lams = sorted({l for _, l, _ in tr})
    assert lams[0] == 1.0 and lams[-1] == 1e4
    assert omsg.stage_tolerance(1e4, 1e-6, 1e-2) == pytest.approx(1e-4, rel=1e-12)
    assert omsg.stage_tolerance(50.0, 1e-6, 1e-2) == pytest.approx(1e-5, rel=1e-12)
    assert omsg.stage_tolerance(3.0, 1e-6, 1e-2) == 1e-6
    assert omsg.stage_tolerance(1e4, 1e-3, 1e-2) == 1e-2
