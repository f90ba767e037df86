"""Oracle spherical-harmonic transforms (ctypes front end of sht_direct.c).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Conventions (shared by the whole oracle):
* maps are FP64 arrays in HEALPix RING order, Npix = 12 nside^2;
* alm are complex128 arrays in m-major order, index m*(2 lmax+1-m)/2 + l,
  for m >= 0 (the real field fixes the negative-m half);
* ``alm2map`` is the real synthesis Y, ``adjoint`` the plain transpose Y^T
  (no weights) written in complex storage, so map2alm = Omega * Y^T with
  Omega = 4 pi / Npix;
* the real orthonormal coefficient vector x has x_l0 = a_l0 and, for m > 0,
  x^c = sqrt(2) Re a_lm, x^s = sqrt(2) Im a_lm; its Euclidean norm is
  sum_l |a_l0|^2 + 2 sum_{m>0} |a_lm|^2 (``alm_dot``).
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        c_int, c_long, c_dbl = ctypes.c_int, ctypes.c_long, ctypes.c_double
        P = ctypes.POINTER
        L.orc_npix.restype = c_long
        L.orc_nalm.restype = c_long
        L.orc_ring_info.argtypes = [c_int, c_int, P(c_long), P(c_int), P(c_dbl),
                                    P(c_dbl), P(c_dbl)]
        for name in ("orc_alm2map", "orc_map2alm_adjoint"):
            getattr(L, name).argtypes = [c_int, c_int, ctypes.c_void_p,
                                         ctypes.c_void_p]
        L.orc_alm2map_pixels.argtypes = [c_int, c_int, ctypes.c_void_p, c_long,
                                         ctypes.c_void_p, ctypes.c_void_p]
        L.orc_map2alm_modes.argtypes = [c_int, c_int, ctypes.c_void_p, c_long,
                                        ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]
        L.orc_ymatrix.argtypes = [c_int, c_int, ctypes.c_void_p]
        L.orc_pix_coords.argtypes = [c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]
        L.orc_lambda_all.argtypes = [c_int, c_dbl, c_dbl, ctypes.c_void_p]
        L.orc_lambda_m.argtypes = [c_int, c_int, c_dbl, c_dbl, ctypes.c_void_p]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    return int(lib().orc_threads())


# ---------------------------------------------------------------- geometry
def npix(nside):
    return 12 * nside * nside


def nalm(lmax):
    return (lmax + 1) * (lmax + 2) // 2


def alm_index(lmax, l, m):
    return m * (2 * lmax + 1 - m) // 2 + l


def lm_arrays(lmax):
    """l and m of every alm slot, in storage order."""
    ls = np.concatenate([np.arange(m, lmax + 1) for m in range(lmax + 1)])
    ms = np.concatenate([np.full(lmax + 1 - m, m) for m in range(lmax + 1)])
    return ls, ms


def ring_info(nside, ring):
    """(first pixel, npix in ring, z, sin theta, phi of first pixel); ring is
    1-based."""
    f, n = ctypes.c_long(), ctypes.c_int()
    z, st, p0 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_ring_info(nside, ring, ctypes.byref(f), ctypes.byref(n),
                        ctypes.byref(z), ctypes.byref(st), ctypes.byref(p0))
    return f.value, n.value, z.value, st.value, p0.value


def pix_coords(nside):
    n = npix(nside)
    z, st, phi = np.empty(n), np.empty(n), np.empty(n)
    lib().orc_pix_coords(nside, _ptr(z), _ptr(st), _ptr(phi))
    return z, st, phi


# ---------------------------------------------------------------- Legendre
def lambda_all(lmax, z, sth):
    out = np.empty(nalm(lmax))
    lib().orc_lambda_all(lmax, float(z), float(sth), _ptr(out))
    return out


def lambda_m(lmax, m, z, sth):
    out = np.empty(lmax + 1 - m)
    lib().orc_lambda_m(lmax, m, float(z), float(sth), _ptr(out))
    return out


# ---------------------------------------------------------------- transforms
def alm2map(alm, nside, lmax):
    """s = Y a (real synthesis), direct sum over all (l, m) at every pixel."""
    a = np.ascontiguousarray(alm, dtype=np.complex128)
    assert a.shape == (nalm(lmax),)
    out = np.empty(npix(nside))
    lib().orc_alm2map(nside, lmax, _ptr(a), _ptr(out))
    return out


def alm2map_pixels(alm, nside, lmax, pix):
    a = np.ascontiguousarray(alm, dtype=np.complex128)
    p = np.ascontiguousarray(pix, dtype=np.int64)
    out = np.empty(len(p))
    lib().orc_alm2map_pixels(nside, lmax, _ptr(a), len(p), _ptr(p), _ptr(out))
    return out


def adjoint(m, nside, lmax):
    """b = Y^T s (no weights), complex storage."""
    s = np.ascontiguousarray(m, dtype=np.float64)
    assert s.shape == (npix(nside),)
    out = np.empty(nalm(lmax), dtype=np.complex128)
    lib().orc_map2alm_adjoint(nside, lmax, _ptr(s), _ptr(out))
    return out


def adjoint_modes(m, nside, lmax, ls, ms):
    s = np.ascontiguousarray(m, dtype=np.float64)
    ls = np.ascontiguousarray(ls, dtype=np.int32)
    ms = np.ascontiguousarray(ms, dtype=np.int32)
    out = np.empty(len(ls), dtype=np.complex128)
    lib().orc_map2alm_modes(nside, lmax, _ptr(s), len(ls), _ptr(ls), _ptr(ms),
                            _ptr(out))
    return out


def map2alm(m, nside, lmax):
    """Omega * Y^T s: the unweighted HEALPix analysis."""
    return (4.0 * np.pi / npix(nside)) * adjoint(m, nside, lmax)


# ---------------------------------------------------------------- real basis
def ymatrix(nside, lmax):
    """Explicit real synthesis matrix Y, shape (Npix, (lmax+1)^2); columns in
    the order of ``alm_to_real``."""
    Y = np.empty((npix(nside), (lmax + 1) ** 2))
    lib().orc_ymatrix(nside, lmax, _ptr(Y))
    return Y


def real_layout(lmax):
    """For every real coefficient: (alm slot, part) with part 0 = m=0 real,
    1 = sqrt(2) Re, 2 = sqrt(2) Im.  Matches the column order of ymatrix."""
    slots, parts = [], []
    for l in range(lmax + 1):
        slots.append(alm_index(lmax, l, 0))
        parts.append(0)
    for m in range(1, lmax + 1):
        for l in range(m, lmax + 1):
            i = alm_index(lmax, l, m)
            slots += [i, i]
            parts += [1, 2]
    return np.array(slots), np.array(parts)


def alm_to_real(alm, lmax):
    slots, parts = real_layout(lmax)
    a = alm[slots]
    return np.where(parts == 0, a.real,
                    np.where(parts == 1, np.sqrt(2) * a.real,
                             np.sqrt(2) * a.imag))


def real_to_alm(x, lmax):
    slots, parts = real_layout(lmax)
    out = np.zeros(nalm(lmax), dtype=np.complex128)
    re = np.zeros(nalm(lmax))
    im = np.zeros(nalm(lmax))
    sel0 = parts == 0
    re[slots[sel0]] = x[sel0]
    re[slots[parts == 1]] = x[parts == 1] / np.sqrt(2)
    im[slots[parts == 2]] = x[parts == 2] / np.sqrt(2)
    out.real, out.imag = re, im
    return out


def real_ell(lmax):
    """l of every real coefficient."""
    slots, _ = real_layout(lmax)
    ls, _ = lm_arrays(lmax)
    return ls[slots]


def alm_weights(lmax):
    """1 for m = 0 slots, 2 for m > 0: the real-basis inner-product weights
    in complex storage."""
    _, ms = lm_arrays(lmax)
    return np.where(ms == 0, 1.0, 2.0)


def alm_dot(a, b, lmax):
    """Real-basis inner product <x_a, x_b> in complex storage."""
    w = alm_weights(lmax)
    return float(np.sum(w * (a.real * b.real + a.imag * b.imag)))


def alm_norm(a, lmax):
    return np.sqrt(alm_dot(a, a, lmax))
