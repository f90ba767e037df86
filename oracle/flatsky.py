"""Oracle for the dual messenger on the flat sky (the paper's Algorithm 2 on
its own Sect. 3 workload: an N x N periodic grid of angular side L, 2-D FFTs).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 numpy.

Conventions and readings (each is listed in the design notes):
* The Fourier transform is the plain 2-D DFT (numpy fft2, with ifft2 its
  inverse).  A pointwise filter commutes with the DFT's normalisation, so
  s = ifft2(f_k fft2(t)) is Algorithm 2's F^-1([.]_k F(t)) for any scaling
  that makes F^-1 F = 1.
* Units: the signal power C_l (l = 2 pi |k| / L) and a pixel variance v
  compare as C_l against v Omega_pix, Omega_pix = (L / N)^2 (the white
  noise of variance v has power v Omega_pix); this is the paper's factor
  sigma = N^2 / L^4 up to the DFT's normalisation, the same reading as on
  the sphere (Omega = pixel solid angle).
* Signal step: t_hat = f_k fft2(t), f_k = Sbar_k / (Sbar_k + xi Omega_pix),
  Sbar_k = max(C_k - mu Omega_pix, 0) (Theta(S - U), App. B); s = ifft2.
* Messenger step (Eq. 14 with Nbar = N - alpha): t = s + xi / (sigma^2 + mu)
  (d - s); the paper's mask is a finite 10^6 N, so no pixel has weight 0.
* Cooling xi <- max(alpha, beta xi), mu = xi - alpha; start mu_0 Omega_pix =
  beta max_k C_k; stage tolerance min(eps_cap, eps max(1, mu / alpha)).
* Cauchy ratio ||s_i - s_{i-1}|| / ||s_i|| on the pixel map (equal to the
  ratio of the DFT coefficients by Parseval).
* Here the basis change is orthogonal, so the last stage's fixed point is
  the Wiener filter of Eq. (2) itself (no quadrature gap).
"""
import numpy as np


def stage_eps(mu, alpha, eps_final, eps_cap):
    if mu == 0.0:
        return eps_final
    return min(eps_cap, eps_final * max(1.0, mu / alpha))


def dual_messenger_flat(d, noise_var, ck, pixel_area, beta=0.75, eps_final=1e-6,
                        eps_cap=1e-2, max_iter=200_000, stop="cauchy", trace=None):
    """Algorithm 2 on the flat sky.  d, noise_var: N x N pixel maps; ck:
    C at each DFT mode (numpy fft2 order).  Returns (s, info)."""
    d = np.asarray(d, dtype=np.float64)
    nv = np.asarray(noise_var, dtype=np.float64)
    om = float(pixel_area)
    alpha = float(np.min(nv))                      # T = alpha 1
    s = np.zeros_like(d)                           # s_0 = 0
    t = d.copy()                                   # t_0 = d
    mu = beta * float(np.max(ck)) / om
    xi = alpha + mu
    it, stage, converged, c = 0, 0, False, 1.0
    while True:
        sbar = np.maximum(ck - mu * om, 0.0)       # Sbar = Theta(S - U)
        f = sbar / (sbar + xi * om)
        w = xi / (nv + mu)
        eps = stage_eps(mu, alpha, eps_final, eps_cap)
        hist, prev_c = [], None
        while True:
            s_new = np.real(np.fft.ifft2(f * np.fft.fft2(t)))   # signal step
            t = s_new + w * (d - s_new)                          # messenger step
            num = np.linalg.norm(s_new - s)
            den = np.linalg.norm(s_new)
            c = num / den if den > 0 else 0.0
            s = s_new
            it += 1
            if trace is not None:
                trace.append((stage, xi, mu, c))
            if mu == 0.0 and stop == "error":
                hist.append(c)
                if len(hist) > 16 and prev_c and c > 0:
                    r = min(max(c / prev_c, (c / hist[-17]) ** (1.0 / 16.0)), 0.999999)
                    if c * r / (1.0 - r) < eps_final:
                        converged = True
                        break
            elif c < eps:
                converged = mu == 0.0
                break
            prev_c = c
            if it >= max_iter:
                break
        if mu == 0.0 or it >= max_iter:
            break
        xi = max(alpha, beta * xi)
        mu = xi - alpha if xi > alpha else 0.0
        stage += 1
    return s, {"iterations": it, "stages": stage + 1, "converged": converged,
               "alpha": alpha, "final_cauchy": c}


def signal_cov_dense(ck, pixel_area):
    """S in the pixel basis: U^H diag(C_k / Omega_pix) U with U the unitary
    2-D DFT (small N only)."""
    n = ck.shape[0]
    F = np.fft.fft(np.eye(n))
    U = np.kron(F, F) / n
    S = U.conj().T @ (np.asarray(ck, dtype=np.float64).ravel()[:, None] / pixel_area * U)
    return np.real(S)


def wf_dense(d, noise_var, ck, pixel_area):
    """Eq. (2) by a dense solve: s = S (S + N)^-1 d (small N only)."""
    S = signal_cov_dense(ck, pixel_area)
    dv = np.asarray(d, dtype=np.float64).ravel()
    sol = np.linalg.solve(S + np.diag(np.asarray(noise_var, dtype=np.float64).ravel()), dv)
    return (S @ sol).reshape(d.shape)


def wf_cg(d, noise_var, ck, pixel_area, tol=1e-12, max_iter=20000):
    """Eq. (2) by conjugate gradients on App. C's form (1 + S^1/2 N^-1 S^1/2) z
    = S^1/2 N^-1 d, s = S^1/2 z, S^1/2 v = ifft2(sqrt(C / Omega) fft2(v)),
    preconditioned by its harmonic diagonal 1 + (C / Omega) mean(N^-1); stops
    on the relative residual.  Returns (s, info)."""
    sq = np.sqrt(np.asarray(ck, dtype=np.float64) / pixel_area)
    ninv = 1.0 / np.asarray(noise_var, dtype=np.float64)
    half = lambda v: np.real(np.fft.ifft2(sq * np.fft.fft2(v)))
    A = lambda z: z + half(ninv * half(z))
    y = half(ninv * d)
    pd = 1.0 + sq ** 2 * float(np.mean(ninv))
    prec = lambda r: np.real(np.fft.ifft2(np.fft.fft2(r) / pd))
    z = np.zeros_like(y)
    r = y.copy()
    q = prec(r)
    p = q.copy()
    rz = float(np.sum(r * q))
    ny = np.linalg.norm(y)
    it, rel = 0, 1.0
    while it < max_iter:
        Ap = A(p)
        a = rz / float(np.sum(p * Ap))
        z = z + a * p
        r = r - a * Ap
        it += 1
        rel = np.linalg.norm(r) / ny
        if rel < tol:
            break
        q = prec(r)
        rz_new = float(np.sum(r * q))
        p = q + (rz_new / rz) * p
        rz = rz_new
    return half(z), {"iterations": it, "rel_residual": rel}
