/*
 * Seeded synthetic inputs for the Wilson-clover operator: SU(3) gauge links and
 * Gaussian spinor fields.
 *
 * This module holds none of the operator's arithmetic.  It only draws inputs,
 * and both the CPU oracle and the CUDA library consume what it produces.
 *
 * Random numbers are counter based, so any site can be generated on its own
 * and the result does not depend on the thread count:
 *   key      = mix64(seed)
 *   word(k)  = mix64(key + (k + 1) * 0x9E3779B97F4A7C15)     (SplitMix64, Steele et al. 2014)
 *   normal pair k: u1 = ((word(2k) >> 11) + 1) * 2^-53 in (0, 1],
 *                  u2 =  (word(2k+1) >> 11)    * 2^-53 in [0, 1),
 *                  (re, im) = sqrt(-2 ln u1) * (cos 2 pi u2, sin 2 pi u2)    (Box-Muller)
 * Each complex entry uses one normal pair, so Re and Im are i.i.d. N(0, 1).
 *
 * Gauge link U_mu(x) for site x (lexicographic, X fastest) and direction mu
 * (0..3 = T, Z, Y, X): pair counters (x * 4 + mu) * 9 + j, j = 0..8, fill a 3x3
 * complex matrix A row-major; H = (A + A^H) / 2 minus (tr H / 3) I is a
 * traceless Hermitian Gaussian matrix and U = exp(i eps H), which is special
 * unitary.  The exponential is taken by scaling and squaring of a 14-term
 * Taylor series (Higham, "The scaling and squaring method for the matrix
 * exponential revisited", 2005), which is exact to rounding for these norms.
 *
 * Spinor component c (0..11, c = 3 * spin + colour) of site x of field r uses
 * pair counter (r * V + x) * 12 + c.
 *
 * Layouts: complex numbers are interleaved (re, im) doubles.
 *   links  [site][mu][3][3]
 *   spinor [r][site][12]
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline uint64_t word_at(uint64_t key, uint64_t k) {
  return mix64(key + (k + 1ULL) * 0x9E3779B97F4A7C15ULL);
}

static inline void normal_pair(uint64_t key, uint64_t pair, double out[2]) {
  const double two53 = 1.0 / 9007199254740992.0; /* 2^-53 */
  double u1 = (double)((word_at(key, 2 * pair) >> 11) + 1ULL) * two53;
  double u2 = (double)(word_at(key, 2 * pair + 1) >> 11) * two53;
  double r = sqrt(-2.0 * log(u1));
  double th = 6.283185307179586476925286766559 * u2;
  out[0] = r * cos(th);
  out[1] = r * sin(th);
}

/* 3x3 complex helpers on interleaved storage m[(3 * a + b) * 2 + {0,1}] */
static void m3_mul(const double* A, const double* B, double* C) {
  double t[18];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double re = 0.0, im = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double* x = A + (3 * a + k) * 2;
        const double* y = B + (3 * k + b) * 2;
        re += x[0] * y[0] - x[1] * y[1];
        im += x[0] * y[1] + x[1] * y[0];
      }
      t[(3 * a + b) * 2] = re;
      t[(3 * a + b) * 2 + 1] = im;
    }
  memcpy(C, t, sizeof t);
}

/* U = exp(X) for a 3x3 complex X (here X = i eps H). */
static void m3_exp(const double* X, double* U) {
  double nrm = 0.0;
  for (int i = 0; i < 18; ++i) nrm += X[i] * X[i];
  nrm = sqrt(nrm);
  int k = 0;
  double scale = 1.0;
  while (nrm * scale > 0.25) {
    scale *= 0.5;
    ++k;
  }
  double Y[18];
  for (int i = 0; i < 18; ++i) Y[i] = X[i] * scale;
  /* Horner: E = I + Y (I + Y/2 (I + Y/3 (... (I + Y/14)))) */
  double E[18] = {0};
  for (int a = 0; a < 3; ++a) E[(4 * a) * 2] = 1.0;
  for (int n = 14; n >= 1; --n) {
    double T[18];
    m3_mul(Y, E, T);
    for (int i = 0; i < 18; ++i) E[i] = T[i] / (double)n;
    for (int a = 0; a < 3; ++a) E[(4 * a) * 2] += 1.0;
  }
  for (int s = 0; s < k; ++s) m3_mul(E, E, E);
  memcpy(U, E, sizeof E);
}

/* One special-unitary matrix exp(i eps H) from pair counters base .. base + 8. */
static void su3_from_counter(uint64_t key, uint64_t base, double eps, double* U) {
  double A[18], H[18], X[18];
  for (int j = 0; j < 9; ++j) normal_pair(key, base + (uint64_t)j, A + 2 * j);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const double* ab = A + (3 * a + b) * 2;
      const double* ba = A + (3 * b + a) * 2;
      H[(3 * a + b) * 2] = 0.5 * (ab[0] + ba[0]);
      H[(3 * a + b) * 2 + 1] = 0.5 * (ab[1] - ba[1]);
    }
  double tr = (H[0] + H[8] + H[16]) / 3.0; /* diagonal is real */
  for (int a = 0; a < 3; ++a) H[(4 * a) * 2] -= tr;
  for (int i = 0; i < 9; ++i) { /* X = i eps H */
    X[2 * i] = -eps * H[2 * i + 1];
    X[2 * i + 1] = eps * H[2 * i];
  }
  m3_exp(X, U);
}

/* Links U_mu(x) for sites [site0, site0 + nsites) and mu < nmu into
 * out[(x - site0)][mu][3][3] (nmu = 4 for a gauge field; nmu = 1 gives one
 * SU(3) matrix per site, used for gauge transformations). */
void synth_links(uint64_t seed, double eps, int64_t site0, int64_t nsites, int nmu, double* out) {
  const uint64_t key = mix64(seed);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nsites; ++i)
    for (int mu = 0; mu < nmu; ++mu) {
      uint64_t link = (uint64_t)(site0 + i) * 4ULL + (uint64_t)mu;
      su3_from_counter(key, link * 9ULL, eps, out + (i * nmu + mu) * 18);
    }
}

/* n complex Gaussian numbers from pair counters counter0 .. counter0 + n - 1. */
void synth_gaussian(uint64_t seed, int64_t counter0, int64_t n, double* out) {
  const uint64_t key = mix64(seed);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) normal_pair(key, (uint64_t)(counter0 + i), out + 2 * i);
}

/* Spinor field r of a lattice with V sites, restricted to a list of sites:
 * out[i][12] = psi_r(sites[i]). */
void synth_spinor_sites(uint64_t seed, int64_t V, int64_t r, const int64_t* sites, int64_t nsites, double* out) {
  const uint64_t key = mix64(seed);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nsites; ++i)
    for (int c = 0; c < 12; ++c)
      normal_pair(key, (uint64_t)((r * V + sites[i]) * 12 + c), out + (i * 12 + c) * 2);
}

/* Links of a list of sites: out[i][mu][3][3] = U_mu(sites[i]). */
void synth_links_sites(uint64_t seed, double eps, const int64_t* sites, int64_t nsites, double* out) {
  const uint64_t key = mix64(seed);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nsites; ++i)
    for (int mu = 0; mu < 4; ++mu) {
      uint64_t link = (uint64_t)sites[i] * 4ULL + (uint64_t)mu;
      su3_from_counter(key, link * 9ULL, eps, out + (i * 4 + mu) * 18);
    }
}
