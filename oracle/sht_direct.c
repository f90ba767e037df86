/*
 * oracle/sht_direct.c -- plain FP64 reference implementation of the HEALPix
 * ring geometry and of the spherical-harmonic synthesis / adjoint written as
 * the direct O(Npix * Nalm) sums.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests/, __graft_entry__.smoke() and the cpu_baseline
 * leg of bench.py use it.  It shares no code with the CUDA path.
 *
 * What it computes (all FP64, Condon-Shortley phase, orthonormal Y_lm):
 *   synthesis   s(p)   = sum_l [ a_l0 lam_l0(z_p)
 *                                + 2 sum_{m>0} Re(a_lm e^{i m phi_p}) lam_lm(z_p) ]
 *   adjoint     b_lm   = sum_p s(p) lam_lm(z_p) e^{-i m phi_p}
 * i.e. the real-field synthesis Y and its plain transpose Y^T (no quadrature
 * weights) in complex alm storage, alm index m*(2*lmax+1-m)/2 + l.
 * The Wiener-filter problem these serve is Eq. (2) of the paper; the signal
 * covariance is diagonal in this harmonic basis (Sect. 2, "basis where S is
 * sparse"), the noise covariance diagonal in the pixel basis.
 *
 * Pixel geometry: the HEALPix RING scheme (Gorski et al. 2005): 4*nside-1
 * iso-latitude rings; north-cap ring i (1 <= i < nside) has 4i pixels at
 * z = 1 - i^2/(3 nside^2), phi = (j + 1/2) pi/(2i); equatorial ring i
 * (nside <= i <= 3 nside) has 4 nside pixels at z = (4/3) - 2i/(3 nside),
 * phi = j pi/(2 nside) when i + nside is odd and (j + 1/2) pi/(2 nside) when
 * it is even; the south cap mirrors the north cap.
 *
 * Normalised associated Legendre functions lam_lm(z) (so that
 * Y_lm = lam_lm(cos theta) e^{i m phi}) come from the textbook recurrences:
 *   lam_00 = 1/sqrt(4 pi),
 *   lam_mm = -sin(theta) sqrt((2m+1)/(2m)) lam_{m-1,m-1},
 *   lam_{m+1,m} = sqrt(2m+3) z lam_mm,
 *   lam_lm = sqrt((4l^2-1)/(l^2-m^2)) (z lam_{l-1,m}
 *            - sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)) lam_{l-2,m}).
 * Values too small for a double are carried as (mantissa, power-of-two
 * exponent) while they are tiny and flushed to the double they represent
 * (possibly 0) when stored.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------ */
/* geometry                                                            */
/* ------------------------------------------------------------------ */

long orc_npix(int nside) { return 12L * nside * nside; }
int orc_nring(int nside) { return 4 * nside - 1; }

/* ring: 1-based ring number (1 .. 4 nside - 1).  Returns the index of the
 * first pixel, the number of pixels, z, sin(theta) and the azimuth of the
 * first pixel. */
void orc_ring_info(int nside, int ring, long *first, int *npix, double *z,
                   double *sth, double *phi0) {
  const double ns = (double)nside;
  int north = ring <= 2 * nside ? ring : 4 * nside - ring; /* mirror */
  int n;
  double zz, st, p0;
  long f;
  if (north < nside) { /* polar cap */
    n = 4 * north;
    double omz = (double)north * north / (3.0 * ns * ns); /* 1 - z */
    zz = 1.0 - omz;
    st = sqrt(omz * (2.0 - omz));
    p0 = ORC_PI / (4.0 * north);
  } else { /* equatorial belt */
    n = 4 * nside;
    zz = (2.0 * ns - north) * 2.0 / (3.0 * ns);
    st = sqrt((1.0 - zz) * (1.0 + zz));
    /* first pixel sits at phi = 0 when (ring + nside) is odd, else half a
     * pixel further */
    p0 = ((ring + nside) & 1) ? 0.0 : ORC_PI / (4.0 * ns);
  }
  if (ring <= 2 * nside) {
    if (ring < nside)
      f = 2L * ring * (ring - 1);
    else
      f = 2L * nside * (nside - 1) + (long)(ring - nside) * 4 * nside;
  } else {
    zz = -zz;
    /* count the pixels from the south pole: rings below have the mirror
     * layout */
    long npx = 12L * nside * nside;
    long after; /* pixels strictly after this ring */
    int sring = 4 * nside - ring; /* ring number counted from the south */
    if (sring < nside)
      after = 2L * sring * (sring - 1);
    else
      after = 2L * nside * (nside - 1) + (long)(sring - nside) * 4 * nside;
    f = npx - after - n;
  }
  *first = f;
  *npix = n;
  *z = zz;
  *sth = st;
  *phi0 = p0;
}

/* z, sin(theta), phi for every pixel in RING order */
void orc_pix_coords(int nside, double *z, double *sth, double *phi) {
  int nr = orc_nring(nside);
  for (int r = 1; r <= nr; ++r) {
    long f;
    int n;
    double zz, st, p0;
    orc_ring_info(nside, r, &f, &n, &zz, &st, &p0);
    for (int j = 0; j < n; ++j) {
      z[f + j] = zz;
      sth[f + j] = st;
      phi[f + j] = p0 + 2.0 * ORC_PI * j / n;
    }
  }
}

/* ------------------------------------------------------------------ */
/* normalised associated Legendre functions                            */
/* ------------------------------------------------------------------ */

static long alm_index(int lmax, int l, int m) {
  return (long)m * (2 * lmax + 1 - m) / 2 + l;
}

long orc_nalm(int lmax) { return (long)(lmax + 1) * (lmax + 2) / 2; }

#define BIG_EXP 400 /* rescale step, powers of two */

/* lam_lm(z) for l = m .. lmax at fixed m, written to out[l - m].
 * The seed lam_mm is built by repeated multiplication with exact power-of-two
 * rescaling, so it keeps full relative precision even when it is far below
 * the double range; the stored value is ldexp(mantissa, exponent). */
void orc_lambda_m(int lmax, int m, double z, double sth, double *out) {
  /* seed */
  double v = 1.0 / sqrt(4.0 * ORC_PI);
  int e = 0;
  for (int k = 1; k <= m; ++k) {
    v *= -sth * sqrt((2.0 * k + 1.0) / (2.0 * k));
    if (v != 0.0 && fabs(v) < 0x1p-400) {
      v = ldexp(v, BIG_EXP);
      e -= BIG_EXP;
    }
  }
  if (m > lmax) return;
  double lm2 = 0.0, lm1 = v; /* lam_{l-2}, lam_{l-1} scaled by 2^-e */
  out[0] = ldexp(v, e);
  for (int l = m + 1; l <= lmax; ++l) {
    double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
    double b = (l - 1 > m)
                   ? sqrt((((double)(l - 1) * (l - 1)) - (double)m * m) /
                          (4.0 * (l - 1) * (l - 1) - 1.0))
                   : 0.0;
    double lv = a * (z * lm1 - b * lm2);
    lm2 = lm1;
    lm1 = lv;
    if (e < 0 && fabs(lm1) > 0x1p+400) {
      lm1 = ldexp(lm1, -BIG_EXP);
      lm2 = ldexp(lm2, -BIG_EXP);
      e += BIG_EXP;
    }
    out[l - m] = ldexp(lm1, e);
  }
}

/* all lam_lm(z), healpy alm order */
void orc_lambda_all(int lmax, double z, double sth, double *out) {
  double *tmp = (double *)malloc(sizeof(double) * (lmax + 1));
  for (int m = 0; m <= lmax; ++m) {
    orc_lambda_m(lmax, m, z, sth, tmp);
    for (int l = m; l <= lmax; ++l) out[alm_index(lmax, l, m)] = tmp[l - m];
  }
  free(tmp);
}

/* ------------------------------------------------------------------ */
/* direct transforms                                                   */
/* ------------------------------------------------------------------ */

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* value of the real field with complex alm (interleaved re,im) at one pixel,
 * given the lam table of its ring */
static double synth_point(int lmax, const double *alm, const double *lam,
                          double phi) {
  double acc = 0.0;
  for (int m = 0; m <= lmax; ++m) {
    double c = cos(m * phi), s = sin(m * phi);
    for (int l = m; l <= lmax; ++l) {
      long i = alm_index(lmax, l, m);
      double re = alm[2 * i], im = alm[2 * i + 1];
      double term = (m == 0) ? re : 2.0 * (re * c - im * s);
      acc += lam[i] * term;
    }
  }
  return acc;
}

/* s = Y a on all pixels */
void orc_alm2map(int nside, int lmax, const double *alm, double *map) {
  int nr = orc_nring(nside);
  long nalm = orc_nalm(lmax);
#pragma omp parallel
  {
    double *lam = (double *)malloc(sizeof(double) * nalm);
#pragma omp for schedule(dynamic, 1)
    for (int r = 1; r <= nr; ++r) {
      long f;
      int n;
      double z, st, p0;
      orc_ring_info(nside, r, &f, &n, &z, &st, &p0);
      orc_lambda_all(lmax, z, st, lam);
      for (int j = 0; j < n; ++j)
        map[f + j] = synth_point(lmax, alm, lam, p0 + 2.0 * ORC_PI * j / n);
    }
    free(lam);
  }
}

/* s = Y a on selected pixels only */
void orc_alm2map_pixels(int nside, int lmax, const double *alm, long nsel,
                        const long *pix, double *out) {
  long nalm = orc_nalm(lmax);
  int nr = orc_nring(nside);
#pragma omp parallel
  {
    double *lam = (double *)malloc(sizeof(double) * nalm);
#pragma omp for schedule(dynamic, 1)
    for (long k = 0; k < nsel; ++k) {
      long p = pix[k];
      /* locate the ring by scanning; tests only */
      for (int r = 1; r <= nr; ++r) {
        long f;
        int n;
        double z, st, p0;
        orc_ring_info(nside, r, &f, &n, &z, &st, &p0);
        if (p >= f && p < f + n) {
          orc_lambda_all(lmax, z, st, lam);
          out[k] = synth_point(lmax, alm, lam,
                               p0 + 2.0 * ORC_PI * (double)(p - f) / n);
          break;
        }
      }
    }
    free(lam);
  }
}

/* b = Y^T s (no weights), complex storage: b_lm = sum_p s_p lam e^{-im phi} */
void orc_map2alm_adjoint(int nside, int lmax, const double *map, double *alm) {
  int nr = orc_nring(nside);
#pragma omp parallel
  {
    double *lam = (double *)malloc(sizeof(double) * (lmax + 1));
#pragma omp for schedule(dynamic, 1)
    for (int m = 0; m <= lmax; ++m) {
      for (int l = m; l <= lmax; ++l) {
        long i = alm_index(lmax, l, m);
        alm[2 * i] = 0.0;
        alm[2 * i + 1] = 0.0;
      }
      for (int r = 1; r <= nr; ++r) {
        long f;
        int n;
        double z, st, p0;
        orc_ring_info(nside, r, &f, &n, &z, &st, &p0);
        orc_lambda_m(lmax, m, z, st, lam);
        for (int j = 0; j < n; ++j) {
          double phi = p0 + 2.0 * ORC_PI * j / n;
          double c = cos(m * phi), s = sin(m * phi), v = map[f + j];
          for (int l = m; l <= lmax; ++l) {
            long i = alm_index(lmax, l, m);
            alm[2 * i] += v * lam[l - m] * c;
            alm[2 * i + 1] -= v * lam[l - m] * s;
          }
        }
      }
    }
    free(lam);
  }
}

/* b = Y^T s for selected modes (l[k], m[k]) only */
void orc_map2alm_modes(int nside, int lmax, const double *map, long nsel,
                       const int *ls, const int *ms, double *out) {
  int nr = orc_nring(nside);
#pragma omp parallel
  {
    double *lam = (double *)malloc(sizeof(double) * (lmax + 1));
#pragma omp for schedule(dynamic, 1)
    for (long k = 0; k < nsel; ++k) {
      int l = ls[k], m = ms[k];
      double re = 0.0, im = 0.0;
      for (int r = 1; r <= nr; ++r) {
        long f;
        int n;
        double z, st, p0;
        orc_ring_info(nside, r, &f, &n, &z, &st, &p0);
        orc_lambda_m(l, m, z, st, lam);
        double lv = lam[l - m];
        for (int j = 0; j < n; ++j) {
          double phi = p0 + 2.0 * ORC_PI * j / n;
          double v = map[f + j];
          re += v * lv * cos(m * phi);
          im -= v * lv * sin(m * phi);
        }
      }
      out[2 * k] = re;
      out[2 * k + 1] = im;
    }
    free(lam);
  }
}

/* Explicit real synthesis matrix, row-major [npix][(lmax+1)^2].
 * Column order: for m = 0, l = 0..lmax (Y_l0); then for each m = 1..lmax and
 * l = m..lmax two columns: sqrt(2) lam cos(m phi) and -sqrt(2) lam sin(m phi).
 * With x_l0 = a_l0, x^c = sqrt(2) Re a_lm, x^s = sqrt(2) Im a_lm the map is
 * Y x, identical to orc_alm2map. */
void orc_ymatrix(int nside, int lmax, double *Y) {
  int nr = orc_nring(nside);
  long ncol = (long)(lmax + 1) * (lmax + 1);
  long nalm = orc_nalm(lmax);
#pragma omp parallel
  {
    double *lam = (double *)malloc(sizeof(double) * nalm);
#pragma omp for schedule(dynamic, 1)
    for (int r = 1; r <= nr; ++r) {
      long f;
      int n;
      double z, st, p0;
      orc_ring_info(nside, r, &f, &n, &z, &st, &p0);
      orc_lambda_all(lmax, z, st, lam);
      for (int j = 0; j < n; ++j) {
        double phi = p0 + 2.0 * ORC_PI * j / n;
        double *row = Y + (f + j) * ncol;
        long c = 0;
        for (int l = 0; l <= lmax; ++l) row[c++] = lam[alm_index(lmax, l, 0)];
        for (int m = 1; m <= lmax; ++m) {
          double cm = cos(m * phi), sm = sin(m * phi);
          for (int l = m; l <= lmax; ++l) {
            double lv = lam[alm_index(lmax, l, m)];
            row[c++] = sqrt(2.0) * lv * cm;
            row[c++] = -sqrt(2.0) * lv * sm;
          }
        }
      }
    }
    free(lam);
  }
}
