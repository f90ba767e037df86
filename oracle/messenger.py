"""Oracle for the standard messenger algorithm (the paper's Algorithm 1,
Sect. 2.1, Eqs. 4-5) on the HEALPix sphere.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 numpy; the
transforms are those of oracle.dm (direct sums, or the explicit matrix for
small Nside).

The messenger field t has covariance T = alpha 1 (alpha = min diag N over
observed pixels) and Nbar = N - T.  With the cooling parameter lambda, one
iteration of Algorithm 1 takes, in the paper's order:
* the signal step (Eq. 5): s = [S^-1 + (lambda T)^-1]^-1 (lambda T)^-1 t,
  done in the harmonic basis;
* the messenger step (Eq. 4): t = [Nbar^-1 + (lambda T)^-1]^-1
  [Nbar^-1 d + (lambda T)^-1 s], done in the pixel basis.

Readings of the paper used here (each is listed in the design notes):
* Units as for Algorithm 2: the flat-sky factor sigma becomes 1/Omega, so
  lambda T has the harmonic equivalent lambda alpha Omega and the signal
  step is s_lm = C_l / (C_l + lambda alpha Omega) (Omega Y^T t)_lm.
* The messenger step is written without dividing by Nbar:
  t = s + lambda alpha / (Nbar_p + lambda alpha) (d - s), weight 0 on masked
  pixels (Nbar = infinity); finite where sigma^2_p = alpha (t = d there).
* Cooling: lambda <- max(1, eta lambda) from lambda_0 = 1e4 (Algorithm 1),
  eta = 3/4 (Sect. 4); the stage with lambda = 1 is the last.
* Stage tolerances in three steps (Sect. 4, values only in Fig. 4):
  100 eps for lambda >= 100, 10 eps for 10 <= lambda < 100, eps below,
  capped at eps_cap.
* s_0 = 0, t_0 = d with masked pixels set to 0; Cauchy ratio on the real
  alm norm, as for Algorithm 2.
"""
import numpy as np

from . import sht
from .dm import alpha_of, make_transforms


def signal_filter(cl, lam, alpha, omega):
    """C_l / (C_l + lambda alpha Omega): Eq. (5) in the harmonic basis."""
    return cl / (cl + lam * alpha * omega)


def messenger_weight(noise_var, mask, lam, alpha):
    """lambda alpha / (Nbar_p + lambda alpha), Nbar = sigma^2 - alpha; zero
    on masked pixels: Eq. (4) as t = s + w (d - s)."""
    nbar = np.asarray(noise_var, dtype=np.float64) - alpha
    w = lam * alpha / (nbar + lam * alpha)
    return np.where(mask, 0.0, w)


def stage_tolerance(lam, eps_final, eps_cap):
    """The three-step tolerance schedule (Sect. 4)."""
    if lam >= 100.0:
        return min(eps_cap, 100.0 * eps_final)
    if lam >= 10.0:
        return min(eps_cap, 10.0 * eps_final)
    return eps_final


def standard_messenger(nside, lmax, cl, noise_var, mask, d, eta=0.75, lambda0=1e4,
                       eps_final=1e-13, eps_cap=1e-2, max_iter=400_000, alpha=None,
                       transforms=None, stop="cauchy", trace=None, stage_callback=None):
    """Run Algorithm 1 to the end of its lambda = 1 stage.

    Returns (alm, info).  ``stop`` = "cauchy" ends the last stage when the
    Cauchy ratio drops below eps_final; "error" ends it when the geometric
    error estimate c_i r / (1 - r) does (r = max(c_i / c_{i-1},
    (c_i / c_{i-16})^(1/16))), for tests that converge to the fixed point.
    ``trace`` (a list) receives (stage, lambda, cauchy) per iteration;
    ``stage_callback(stage, lambda, alm)`` is called at the end of each stage."""
    T = transforms if transforms is not None else make_transforms(nside, lmax)
    om = T.omega
    ls, _ = sht.lm_arrays(lmax)
    cl = np.asarray(cl, dtype=np.float64)
    mask = np.asarray(mask, dtype=bool)
    dd = np.where(mask, 0.0, np.asarray(d, dtype=np.float64))
    a = alpha_of(noise_var, mask) if alpha is None else float(alpha)
    s_alm = np.zeros(sht.nalm(lmax), dtype=np.complex128)   # s_0 = 0
    t = dd.copy()                                           # t_0 = d
    lam = float(lambda0)
    it, stage, converged, c = 0, 0, False, 1.0
    while True:
        f = signal_filter(cl, lam, a, om)[ls]
        w = messenger_weight(noise_var, mask, lam, a)
        eps = stage_tolerance(lam, eps_final, eps_cap)
        hist, prev_c = [], None
        while True:
            s_new = f * (om * T.adjoint(t))      # signal step, harmonic basis
            s_map = T.synth(s_new)               # back to the pixel basis
            t = s_map + w * (dd - s_map)         # messenger step
            num = sht.alm_norm(s_new - s_alm, lmax)
            den = sht.alm_norm(s_new, lmax)
            c = num / den if den > 0 else 0.0
            s_alm = s_new
            it += 1
            if trace is not None:
                trace.append((stage, lam, c))
            if lam == 1.0 and stop == "error":
                hist.append(c)
                if len(hist) > 16 and prev_c and c > 0:
                    r = min(max(c / prev_c, (c / hist[-17]) ** (1.0 / 16.0)), 0.999999)
                    if c * r / (1.0 - r) < eps_final:
                        converged = True
                        break
            elif c < eps:
                converged = lam == 1.0
                break
            prev_c = c
            if it >= max_iter:
                break
        if stage_callback is not None:
            stage_callback(stage, lam, s_alm.copy())
        if lam == 1.0 or it >= max_iter:
            break
        lam = max(1.0, eta * lam)
        stage += 1
    return s_alm, {"iterations": it, "stages": stage + 1, "converged": converged,
                   "alpha": a, "final_cauchy": c}


def messenger_fixed_point_dense(nside, lmax, cl, noise_var, mask, d, lam, alpha=None,
                                Y=None):
    """Fixed point of Algorithm 1's inner loop at a given lambda, by a dense
    solve: s = F Omega Y^T [(1 - W) Y s + W d]  <=>
    [1 - F Omega Y^T (1 - W) Y] s = F Omega Y^T W d.  Returns complex alm."""
    Y = sht.ymatrix(nside, lmax) if Y is None else Y
    ell = sht.real_ell(lmax)
    c = np.asarray(cl, dtype=np.float64)[ell]
    om = 4.0 * np.pi / sht.npix(nside)
    a = alpha_of(noise_var, mask) if alpha is None else alpha
    f = signal_filter(c, lam, a, om)
    w = messenger_weight(noise_var, mask, lam, a)
    dd = np.where(mask, 0.0, d)
    M = np.eye(Y.shape[1]) - (f[:, None] * om) * (Y.T @ ((1.0 - w)[:, None] * Y))
    rhs = f * om * (Y.T @ (w * dd))
    return sht.real_to_alm(np.linalg.solve(M, rhs), lmax)
