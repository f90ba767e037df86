"""Seeded synthetic inputs for the dual messenger Wiener filter.

This module is the one piece shared by the CUDA path's tests/benchmark and by
the CPU oracle's tests.  It draws random numbers and builds the problem
definition (spectrum, noise variances, mask, random harmonic coefficients);
it holds none of the solver's arithmetic and no spherical-harmonic transform
(a signal map is made by whoever consumes the coefficients).

Recipe (the paper's Sect. 3 workload moved to the sphere):
* C_l = A / (l (l+1)) b_l^2 for l >= 2, C_0 = C_1 = 0; Gaussian beam
  b_l = exp(-l(l+1) sigma_b^2 / 2), sigma_b = FWHM / sqrt(8 ln 2), FWHM =
  3 pixel widths = 3 sqrt(Omega).
* Signal coefficients: a_l0 ~ N(0, C_l), Re/Im a_lm ~ N(0, C_l / 2) (m > 0).
* "galactic" latitude b is measured from the HEALPix equator; a band mask is
  |b| < b0; point-source discs have uniformly drawn centres.
* Ecliptic frame: the galactic frame rotated by 60.2 deg about the x axis.
* Scan hits: clip(1/|cos beta_ecl|, 1, 100) times a seeded low-order
  azimuthal modulation, clipped again to [1, 100]; sigma^2 = sigma0^2 <h>/h.
* Lognormal noise: sigma^2 = sigma0^2 exp(0.5 g), g ~ N(0, 1).
* sigma0^2 = C_l* b_l*^2 / Omega (signal-to-noise one at l*).
* A masked pixel carries d = 0; its noise variance is irrelevant (N^-1 = 0).
"""
from dataclasses import dataclass, field
import numpy as np

ECLIPTIC_TILT_DEG = 60.2


# ---------------------------------------------------------------- basics
def npix(nside):
    return 12 * nside * nside


def nalm(lmax):
    return (lmax + 1) * (lmax + 2) // 2


def omega(nside):
    return 4.0 * np.pi / npix(nside)


def lm_of_slots(lmax):
    ls = np.concatenate([np.arange(m, lmax + 1) for m in range(lmax + 1)])
    ms = np.concatenate([np.full(lmax + 1 - m, m) for m in range(lmax + 1)])
    return ls, ms


def pixel_centres(nside):
    """(z, phi) of every pixel centre, HEALPix RING order (pixel layout of
    Gorski et al. 2005), used to place masks and scan patterns."""
    n = nside
    zs, ps = [], []
    for ring in range(1, 4 * n):
        north = ring if ring <= 2 * n else 4 * n - ring
        if north < n:
            cnt = 4 * north
            z = 1.0 - north * north / (3.0 * n * n)
            p0 = np.pi / (4.0 * north)
        else:
            cnt = 4 * n
            z = (2 * n - north) * 2.0 / (3.0 * n)
            p0 = 0.0 if (ring + n) % 2 == 1 else np.pi / (4.0 * n)
        if ring > 2 * n:
            z = -z
        zs.append(np.full(cnt, z))
        ps.append(p0 + 2.0 * np.pi * np.arange(cnt) / cnt)
    return np.concatenate(zs), np.concatenate(ps)


def unit_vectors(nside):
    z, phi = pixel_centres(nside)
    st = np.sqrt(np.maximum(0.0, (1.0 - z) * (1.0 + z)))
    return np.stack([st * np.cos(phi), st * np.sin(phi), z], axis=1)


# ---------------------------------------------------------------- spectrum
def beam_fwhm(nside, pixels=3.0):
    return pixels * np.sqrt(omega(nside))


def cl_spectrum(lmax, nside, amplitude=1.0, fwhm=None):
    """C_l = A / (l(l+1)) b_l^2, l >= 2; zero for l < 2."""
    fwhm = beam_fwhm(nside) if fwhm is None else fwhm
    sb = fwhm / np.sqrt(8.0 * np.log(2.0))
    l = np.arange(lmax + 1, dtype=np.float64)
    cl = np.zeros(lmax + 1)
    cl[2:] = amplitude / (l[2:] * (l[2:] + 1.0)) * np.exp(-l[2:] * (l[2:] + 1.0) * sb * sb)
    return cl


def random_alm(rng, cl):
    """Gaussian harmonic coefficients with variance C_l (complex storage)."""
    lmax = len(cl) - 1
    ls, ms = lm_of_slots(lmax)
    var = cl[ls]
    re = rng.standard_normal(len(ls))
    im = rng.standard_normal(len(ls))
    a = np.where(ms == 0, np.sqrt(var) * re, np.sqrt(var / 2.0) * re) \
        + 1j * np.where(ms == 0, 0.0, np.sqrt(var / 2.0) * im)
    return a.astype(np.complex128)


# ---------------------------------------------------------------- masks
def band_mask(nside, b0_deg):
    z, _ = pixel_centres(nside)
    return np.abs(z) < np.sin(np.deg2rad(b0_deg))


def disc_mask(nside, rng, count, radius_deg):
    z, phi = pixel_centres(nside)
    m = np.zeros(len(z), dtype=bool)
    if count == 0:
        return m
    cz = rng.uniform(-1.0, 1.0, count)
    cp = rng.uniform(0.0, 2.0 * np.pi, count)
    r = np.deg2rad(radius_deg)
    cosr = np.cos(r)
    th = np.arccos(cz)
    # pixels are ordered by decreasing z: test only the z-range of each disc
    negz = -z
    for k in range(count):
        zhi = np.cos(max(th[k] - r, 0.0))
        zlo = np.cos(min(th[k] + r, np.pi))
        a = np.searchsorted(negz, -zhi, side="left")
        b = np.searchsorted(negz, -zlo, side="right")
        zz = z[a:b]
        st = np.sqrt(np.maximum(0.0, (1.0 - zz) * (1.0 + zz)))
        cs = np.sqrt(max(0.0, 1.0 - cz[k] * cz[k]))
        dot = st * cs * np.cos(phi[a:b] - cp[k]) + zz * cz[k]
        m[a:b] |= dot > cosr
    return m


def band_for_fraction(nside, target, disc):
    """Smallest band half-width (deg) whose union with ``disc`` masks at least
    ``target`` of the sky."""
    z, _ = pixel_centres(nside)
    lo, hi = 0.0, 90.0
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        frac = np.mean((np.abs(z) < np.sin(np.deg2rad(mid))) | disc)
        lo, hi = (mid, hi) if frac < target else (lo, mid)
    return hi


# ---------------------------------------------------------------- noise
def ecliptic_latitude(nside):
    v = unit_vectors(nside)
    e = np.deg2rad(ECLIPTIC_TILT_DEG)
    # rotate about x: z' = sin(e) y + cos(e) z
    ze = np.sin(e) * v[:, 1] + np.cos(e) * v[:, 2]
    ye = np.cos(e) * v[:, 1] - np.sin(e) * v[:, 2]
    return np.arcsin(np.clip(ze, -1.0, 1.0)), np.arctan2(ye, v[:, 0])


def scan_hits(nside, rng):
    beta, lam = ecliptic_latitude(nside)
    h = 1.0 / np.maximum(np.abs(np.cos(beta)), 1e-6)
    h = np.clip(h, 1.0, 100.0)
    mod = np.ones_like(h)
    for k in range(1, 4):
        amp = 0.15 * rng.standard_normal()
        ph = rng.uniform(0.0, 2.0 * np.pi)
        mod += amp * np.cos(k * lam + ph)
    return np.clip(h * np.clip(mod, 0.2, None), 1.0, 100.0)


def sigma0_sq(cl, nside, ell_star):
    """sigma0^2 with C_l* b_l*^2 = Omega sigma0^2 (signal-to-noise one)."""
    return float(cl[ell_star]) / omega(nside)


# ---------------------------------------------------------------- problems
@dataclass
class Problem:
    """One Wiener-filter problem: spectrum, noise, mask, true signal alm and
    the noise realisation.  The data map is d = Y a_true + n (masked -> 0);
    Y a_true is left to the consumer."""
    nside: int
    lmax: int
    cl: np.ndarray
    noise_var: np.ndarray
    mask: np.ndarray
    alm_true: np.ndarray
    noise: np.ndarray
    seed: int
    name: str = ""
    meta: dict = field(default_factory=dict)

    def data(self, signal_map):
        d = np.asarray(signal_map, dtype=np.float64) + self.noise
        return np.where(self.mask, 0.0, d)


def _finish(nside, lmax, cl, var, mask, rng, seed, name, meta):
    a = random_alm(rng, cl)
    n = np.sqrt(var) * rng.standard_normal(npix(nside))
    var = np.where(mask, 1.0, var)  # arbitrary positive placeholder
    return Problem(nside, lmax, cl, var, mask, a, np.where(mask, 0.0, n), seed,
                   name, meta)


def lognormal_problem(nside, lmax=None, seed=0, band_deg=15.0, discs=20,
                      disc_radius_deg=1.5, ell_star=None, amplitude=1.0):
    """Lognormal per-pixel noise, band + disc mask (the Nside-32 workload:
    |b| < 15 deg band and 20 discs of 3 deg diameter)."""
    lmax = 2 * nside if lmax is None else lmax
    rng = np.random.default_rng(seed)
    cl = cl_spectrum(lmax, nside, amplitude)
    ls_ = lmax // 2 if ell_star is None else ell_star
    s0 = sigma0_sq(cl, nside, ls_)
    var = s0 * np.exp(0.5 * rng.standard_normal(npix(nside)))
    mask = band_mask(nside, band_deg) | disc_mask(nside, rng, discs, disc_radius_deg)
    return _finish(nside, lmax, cl, var, mask, rng, seed, "lognormal",
                   {"sigma0_sq": s0, "ell_star": ls_})


def scan_problem(nside, lmax=None, seed=0, mask_fraction=0.25, discs=500,
                 disc_radius_deg=0.5, ell_star=None, amplitude=1.0):
    """Ecliptic-scan noise (hits 1-100), galactic band tuned so band + discs
    mask ``mask_fraction`` of the sky (the Nside-256 / 1024 workloads)."""
    lmax = 2 * nside if lmax is None else lmax
    rng = np.random.default_rng(seed)
    cl = cl_spectrum(lmax, nside, amplitude)
    if ell_star is None:
        ell_star = min(1000, lmax // 2)
    s0 = sigma0_sq(cl, nside, ell_star)
    hits = scan_hits(nside, rng)
    var = s0 * np.mean(hits) / hits
    disc = disc_mask(nside, rng, discs, disc_radius_deg)
    b0 = band_for_fraction(nside, mask_fraction, disc)
    mask = band_mask(nside, b0) | disc
    return _finish(nside, lmax, cl, var, mask, rng, seed, "scan",
                   {"sigma0_sq": s0, "ell_star": ell_star, "band_deg": b0,
                    "hits_min": float(hits.min()), "hits_max": float(hits.max())})


def uniform_problem(nside, lmax=None, seed=0, sigma_sq=None, amplitude=1.0):
    """Unmasked sky with uniform noise (the closed-form case)."""
    lmax = 2 * nside if lmax is None else lmax
    rng = np.random.default_rng(seed)
    cl = cl_spectrum(lmax, nside, amplitude)
    s0 = sigma0_sq(cl, nside, lmax // 2) if sigma_sq is None else sigma_sq
    var = np.full(npix(nside), s0)
    mask = np.zeros(npix(nside), dtype=bool)
    return _finish(nside, lmax, cl, var, mask, rng, seed, "uniform",
                   {"sigma0_sq": s0})


def batch_problems(count=64, seed_base=3000, nsides=(64, 128, 256)):
    """Uneven batch: Nside drawn from ``nsides``, lmax = 2 Nside, amplitude
    A x U[0.5, 2], scan noise, mask fraction U[5%, 40%]."""
    rng = np.random.default_rng(seed_base)
    out = []
    for i in range(count):
        ns = int(rng.choice(nsides))
        amp = float(rng.uniform(0.5, 2.0))
        frac = float(rng.uniform(0.05, 0.40))
        ndisc = int(rng.integers(0, 60))
        out.append(scan_problem(ns, seed=seed_base + i + 1, mask_fraction=frac,
                                discs=ndisc, disc_radius_deg=0.5,
                                amplitude=amp))
    return out


def random_map(nside, seed):
    return np.random.default_rng(seed).standard_normal(npix(nside))


# ---------------------------------------------------------------- flat sky
# The paper's Sect. 3 workload: an n x n periodic grid of side L = 10 deg,
# white noise of 64 muK^2 with a central 5 deg square at 10^6 times that;
# an analytic spectrum stands in for CAMB.

def flat_mode_ell(n, side):
    """|l| = 2 pi |k| / L of every DFT mode (numpy fft2 order)."""
    k = np.fft.fftfreq(n, d=1.0 / n)
    kx, ky = np.meshgrid(k, k)
    return 2.0 * np.pi * np.hypot(kx, ky) / side


def flat_cl(ell, amplitude=5000.0, ell_damp=1500.0):
    """Analytic stand-in for the paper's CAMB spectrum (muK^2 sr):
    C_l = 2 pi A / (l (l + 1)) exp(-(l / l_d)^2), A the plateau of
    l (l + 1) C_l / 2 pi; C_0 = 0 (no monopole)."""
    ell = np.asarray(ell, dtype=np.float64)
    c = np.zeros_like(ell)
    pos = ell > 0
    e = ell[pos]
    c[pos] = 2.0 * np.pi * amplitude / (e * (e + 1.0)) * np.exp(-(e / ell_damp) ** 2)
    return c


def flat_paper_noise(n, side_deg=10.0, mask_deg=5.0, var=64.0, mask_factor=1e6):
    """White noise of variance 64 muK^2, a central square of side 5 deg
    with 10^6 times that (the Sect. 3 workload)."""
    x = (np.arange(n) + 0.5) * side_deg / n - side_deg / 2.0
    inside = np.abs(x) < mask_deg / 2.0
    m = inside[:, None] & inside[None, :]
    return np.where(m, var * mask_factor, var), m


def flat_gaussian_field(rng, ck, pixel_area):
    """A real Gaussian field whose DFT modes have power C_k / Omega_pix per
    unit white variance (the filter's units): s = ifft2(sqrt(C_k / Omega) *
    fft2(white)), white ~ N(0, 1) per pixel."""
    n = ck.shape[0]
    w = rng.standard_normal((n, n))
    return np.real(np.fft.ifft2(np.sqrt(ck / pixel_area) * np.fft.fft2(w)))
