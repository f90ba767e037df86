"""Oracle for the hybrid dual messenger Wiener filter (the paper's Algorithm 2)
on the HEALPix sphere, and the plain solves it is pinned against.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 numpy; the
spherical-harmonic transforms are the direct sums of oracle.sht (or, for small
Nside, the same operator as an explicit matrix).

Problem (Eq. 1-2): d = s + n, (S^-1 + N^-1) s_WF = N^-1 d, with S diagonal in
the harmonic basis (C_l, isotropic) and N diagonal in the pixel basis
(sigma^2_p; a masked pixel has N^-1 = 0).

Readings of the paper used here (each is listed in the design notes):
* Omega = 4 pi / Npix converts pixel variances to harmonic ones: the flat-sky
  factor sigma of Algorithm 2 becomes 1/Omega.  xi and mu are pixel variances,
  their harmonic equivalents xi*Omega, mu*Omega.
* Signal step (Eq. 15 / Algorithm 2): x <- f_l * (Omega Y^T t) with
  f_l = Sbar_l / (Sbar_l + xi Omega), Sbar_l = max(C_l - mu Omega, 0): the
  truncation Theta(S - U) of App. B.
* Messenger step (Eq. 14, with Nbar = N - alpha): t <- s + w (d - s),
  w_p = xi / (sigma^2_p + mu) (0 on masked pixels), which is
  (Nbar^-1 + xi^-1)^-1 (Nbar^-1 d + xi^-1 s) written without divisions by
  Nbar (so it stays finite where sigma^2_p = alpha).
* Cooling: xi <- max(alpha, beta xi), mu = xi - alpha; the stage with mu = 0
  is the last.  Start: mu_0 Omega = beta max_l C_l.
* Stage tolerance: eps_k = min(eps_cap, eps_final max(1, mu_k / alpha)),
  eps_final for the last stage; Cauchy norm in the real alm basis.
* The initial messenger field is d with masked pixels set to 0; s_0 = 0.
"""
import numpy as np

from . import sht


# ---------------------------------------------------------------- transforms
class DirectTransforms:
    """Y and Y^T via the direct C sums (any Nside)."""

    def __init__(self, nside, lmax):
        self.nside, self.lmax = nside, lmax
        self.omega = 4.0 * np.pi / sht.npix(nside)

    def synth(self, alm):
        return sht.alm2map(alm, self.nside, self.lmax)

    def adjoint(self, m):
        return sht.adjoint(m, self.nside, self.lmax)


class MatrixTransforms:
    """The same operators as an explicit real matrix (small Nside only)."""

    def __init__(self, nside, lmax, Y=None):
        self.nside, self.lmax = nside, lmax
        self.omega = 4.0 * np.pi / sht.npix(nside)
        self.Y = sht.ymatrix(nside, lmax) if Y is None else Y

    def synth(self, alm):
        return self.Y @ sht.alm_to_real(alm, self.lmax)

    def adjoint(self, m):
        return sht.real_to_alm(self.Y.T @ m, self.lmax)


def make_transforms(nside, lmax):
    if sht.npix(nside) * (lmax + 1) ** 2 <= 60_000_000:
        return MatrixTransforms(nside, lmax)
    return DirectTransforms(nside, lmax)


# ---------------------------------------------------------------- pieces
def alpha_of(noise_var, mask):
    """alpha = min diag(N) over observed pixels (Algorithm 2, T = alpha 1)."""
    return float(np.min(noise_var[~mask]))


def filter_ell(cl, xi, mu, omega):
    """f_l = Sbar_l / (Sbar_l + xi Omega), Sbar_l = Theta(C_l - mu Omega)."""
    sbar = np.maximum(cl - mu * omega, 0.0)
    return sbar / (sbar + xi * omega)


def pixel_weight(noise_var, mask, xi, mu):
    """w_p = xi / (sigma^2_p + mu) = xi (Nbar + xi)^-1, zero where masked."""
    w = xi / (noise_var + mu)
    return np.where(mask, 0.0, w)


def stage_eps(mu, alpha, eps_final, eps_cap):
    if mu == 0.0:
        return eps_final
    return min(eps_cap, eps_final * max(1.0, mu / alpha))


def initial_mu(cl, omega, beta):
    return beta * float(np.max(cl)) / omega


# ---------------------------------------------------------------- Algorithm 2
def dual_messenger(nside, lmax, cl, noise_var, mask, d, beta=0.75,
                   eps_final=1e-13, eps_cap=1e-2, max_iter=200_000, mu0=None,
                   alpha=None, transforms=None, stop="cauchy",
                   stage_callback=None, trace=None):
    """Run the hybrid dual messenger to the end of its last stage.

    Returns (alm, info).  ``stop`` = "cauchy" ends the last stage when the
    Cauchy ratio drops below eps_final; "error" ends it when the geometric
    error estimate c_i * r/(1-r) does, r = max(c_i / c_{i-1},
    (c_i / c_{i-16})^(1/16)).
    ``stage_callback(stage, xi, mu, alm)`` is called at the end of each
    stage; ``trace`` (a list) receives (stage, xi, mu, cauchy) per iteration.
    """
    T = transforms if transforms is not None else make_transforms(nside, lmax)
    om = T.omega
    ls, _ = sht.lm_arrays(lmax)
    cl = np.asarray(cl, dtype=np.float64)
    noise_var = np.asarray(noise_var, dtype=np.float64)
    mask = np.asarray(mask, dtype=bool)
    dd = np.where(mask, 0.0, np.asarray(d, dtype=np.float64))
    a = alpha_of(noise_var, mask) if alpha is None else float(alpha)

    x = np.zeros(sht.nalm(lmax), dtype=np.complex128)   # s_0 = 0
    t = dd.copy()                                        # t_0 = d
    mu = initial_mu(cl, om, beta) if mu0 is None else float(mu0)
    xi = a + mu
    it, stage = 0, 0
    converged = False
    while True:
        f = filter_ell(cl, xi, mu, om)[ls]
        w = pixel_weight(noise_var, mask, xi, mu)
        eps = stage_eps(mu, a, eps_final, eps_cap)
        prev_c = None
        hist = []
        while True:
            x_new = f * (om * T.adjoint(t))
            s = T.synth(x_new)
            t = s + w * (dd - s)
            num = sht.alm_norm(x_new - x, lmax)
            den = sht.alm_norm(x_new, lmax)
            c = num / den if den > 0 else 0.0
            x = x_new
            it += 1
            if trace is not None:
                trace.append((stage, xi, mu, c))
            if mu == 0.0 and stop == "error":
                # last stage: stop on the geometric error estimate c r/(1-r);
                # r is the larger of the last ratio and the mean ratio over
                # 16 iterations, so at least 17 iterations are needed
                hist.append(c)
                if len(hist) > 16 and prev_c and c > 0:
                    r = max(c / prev_c, (c / hist[-17]) ** (1.0 / 16.0))
                    r = min(r, 0.999999)
                    if c * r / (1.0 - r) < eps_final:
                        converged = True
                        break
            elif c < eps:
                converged = mu == 0.0
                break
            prev_c = c
            if it >= max_iter:
                break
        if stage_callback is not None:
            stage_callback(stage, xi, mu, x.copy())
        if mu == 0.0 or it >= max_iter:
            break
        xi = max(a, beta * xi)
        mu = xi - a if xi > a else 0.0
        stage += 1
    return x, {"iterations": it, "stages": stage + 1, "converged": converged,
               "alpha": a, "final_cauchy": c}


def dm_iterate(x, nside, lmax, cl, noise_var, mask, d, xi, mu, transforms):
    """One iteration G(x) of Algorithm 2's inner loop at fixed (xi, mu),
    starting from the messenger field consistent with x (t = s + w(d - s),
    s = Y x).  Used for the fixed-point residual ||G(x) - x|| / ||x||."""
    T = transforms
    om = T.omega
    ls, _ = sht.lm_arrays(lmax)
    dd = np.where(mask, 0.0, d)
    s = T.synth(x)
    t = s + pixel_weight(noise_var, mask, xi, mu) * (dd - s)
    return filter_ell(cl, xi, mu, om)[ls] * (om * T.adjoint(t))


# ---------------------------------------------------------------- dense solves
def _real_ops(nside, lmax, cl, noise_var, mask, Y=None):
    Y = sht.ymatrix(nside, lmax) if Y is None else Y
    ell = sht.real_ell(lmax)
    return Y, ell, np.asarray(cl, dtype=np.float64)[ell]


def dm_fixed_point_dense(nside, lmax, cl, noise_var, mask, d, mu, alpha=None,
                         Y=None):
    """Fixed point of Algorithm 2's inner loop at a given mu, by a dense solve:
    x = F Omega Y^T [(1 - W) Y x + W d]  <=>
    [1 - F Omega Y^T (1 - W) Y] x = F Omega Y^T W d.   Returns complex alm."""
    Y, ell, c = _real_ops(nside, lmax, cl, noise_var, mask, Y)
    om = 4.0 * np.pi / sht.npix(nside)
    a = alpha_of(noise_var, mask) if alpha is None else alpha
    xi = a + mu
    f = filter_ell(c, xi, mu, om)
    w = pixel_weight(noise_var, mask, xi, mu)
    dd = np.where(mask, 0.0, d)
    K = Y.shape[1]
    M = np.eye(K) - (f[:, None] * om) * (Y.T @ ((1.0 - w)[:, None] * Y))
    rhs = f * om * (Y.T @ (w * dd))
    return sht.real_to_alm(np.linalg.solve(M, rhs), lmax)


def wf_exact_dense(nside, lmax, cl, noise_var, mask, d, Y=None):
    """Exact Wiener filter, Eq. (2), in the symmetric form of App. C:
    (1 + C^1/2 Y^T N^-1 Y C^1/2) z = C^1/2 Y^T N^-1 d,  x = C^1/2 z."""
    Y, ell, c = _real_ops(nside, lmax, cl, noise_var, mask, Y)
    ninv = np.where(mask, 0.0, 1.0 / noise_var)
    dd = np.where(mask, 0.0, d)
    sq = np.sqrt(c)
    A = np.eye(Y.shape[1]) + sq[:, None] * (Y.T @ (ninv[:, None] * Y)) * sq[None, :]
    y = sq * (Y.T @ (ninv * dd))
    z = np.linalg.solve(A, y)
    return sht.real_to_alm(sq * z, lmax)


# ---------------------------------------------------------------- diagnostics
def wf_residual(alm, nside, lmax, cl, noise_var, mask, d, transforms):
    """||A x - y|| / ||y|| with A = 1 + C^1/2 Y^T N^-1 Y C^1/2, x = C^-1/2 s,
    y = C^1/2 Y^T N^-1 d (App. C); the residual the paper plots in Fig. 5."""
    T = transforms
    ls, _ = sht.lm_arrays(lmax)
    c = np.asarray(cl, dtype=np.float64)[ls]
    ninv = np.where(mask, 0.0, 1.0 / noise_var)
    dd = np.where(mask, 0.0, d)
    sq = np.sqrt(c)
    z = np.where(c > 0, alm / np.where(c > 0, sq, 1.0), 0.0)
    az = z + sq * T.adjoint(ninv * T.synth(sq * z))
    y = sq * T.adjoint(ninv * dd)
    return sht.alm_norm(az - y, lmax) / sht.alm_norm(y, lmax)


def chi2(alm, nside, lmax, cl, noise_var, mask, d, transforms):
    """chi^2 = (d - Y x)^T N^-1 (d - Y x) + x^T C^-1 x (posterior -2 log P)."""
    T = transforms
    ls, _ = sht.lm_arrays(lmax)
    c = np.asarray(cl, dtype=np.float64)[ls]
    ninv = np.where(mask, 0.0, 1.0 / noise_var)
    r = np.where(mask, 0.0, d) - T.synth(alm)
    prior_w = np.where(c > 0, 1.0 / np.where(c > 0, c, 1.0), 0.0)
    w = sht.alm_weights(lmax)
    prior = float(np.sum(w * prior_w * np.abs(alm) ** 2))
    return float(np.sum(ninv * r * r)) + prior


def fixed_point_residual(alm, nside, lmax, cl, noise_var, mask, d, transforms,
                         alpha=None):
    """||G(x) - x|| / ||x|| for the last stage (xi = alpha, mu = 0)."""
    a = alpha_of(noise_var, mask) if alpha is None else alpha
    g = dm_iterate(alm, nside, lmax, cl, noise_var, mask, d, a, 0.0, transforms)
    return sht.alm_norm(g - alm, lmax) / sht.alm_norm(alm, lmax)


# ---------------------------------------------------------------- PCG (App. C)
def pcg_wf(nside, lmax, cl, noise_var, mask, d, tol=1e-12, max_iter=20000,
           restart=200, transforms=None, stop="residual"):
    """Exact Wiener filter by conjugate gradients on App. C's system
    (1 + C^1/2 Y^T N^-1 Y C^1/2) z = C^1/2 Y^T N^-1 d, preconditioned by the
    harmonic diagonal M^-1 = 1 + C_l sum_p N^-1_p / (4 pi) (App. C's
    preconditioner on the sphere), restarted every ``restart`` iterations.
    Stops when ||A z - y|| / ||y|| < tol (``stop`` = "residual"), or on App.
    C's own criterion ||z_{i+1} - z_i|| / ||z_{i+1}|| < tol ("cauchy").
    Returns complex alm x = C^1/2 z."""
    T = transforms if transforms is not None else make_transforms(nside, lmax)
    ls, _ = sht.lm_arrays(lmax)
    c = np.asarray(cl, dtype=np.float64)[ls]
    ninv = np.where(mask, 0.0, 1.0 / noise_var)
    dd = np.where(mask, 0.0, d)
    sq = np.sqrt(c)
    dot = lambda u, v: sht.alm_dot(u, v, lmax)

    def A(z):
        return z + sq * T.adjoint(ninv * T.synth(sq * z))

    y = sq * T.adjoint(ninv * dd)
    ny = np.sqrt(dot(y, y))
    pdiag = 1.0 + c * float(np.sum(ninv)) / (4.0 * np.pi)
    z = np.zeros_like(y)
    it = 0
    rel = cauchy = 1.0
    while it < max_iter:
        r = y - A(z)
        p = r / pdiag
        rz = dot(r, p)
        for _ in range(restart):
            Ap = A(p)
            alpha_k = rz / dot(p, Ap)
            z = z + alpha_k * p
            r = r - alpha_k * Ap
            it += 1
            rel = np.sqrt(dot(r, r)) / ny
            cauchy = abs(alpha_k) * np.sqrt(dot(p, p)) / np.sqrt(dot(z, z))
            if (cauchy if stop == "cauchy" else rel) < tol or it >= max_iter:
                break
            q = r / pdiag
            rz_new = dot(r, q)
            p = q + (rz_new / rz) * p
            rz = rz_new
        if (cauchy if stop == "cauchy" else rel) < tol:
            break
    return sq * z, {"iterations": it, "rel_residual": rel, "cauchy": cauchy}
