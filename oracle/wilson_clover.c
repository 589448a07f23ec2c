/*
 * CPU oracle for the Wilson-clover Dirac operator (plain C99, complex double).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this file; the product path never does.  It shares
 * no code with the CUDA library.
 *
 * It follows the thesis "Accelerating Lattice QCD Simulations using GPUs"
 * (Matthaei, 2023), Section 1.1, term by term and without any of the GPU
 * design's tricks (no half-spinors, no even-odd ordering, no block structure):
 *   - spinor component index 3*spin + colour                       (Eq. 1.2)
 *   - directions T, Z, Y, X = 0, 1, 2, 3; lexicographic sites,
 *     X fastest: site = ((t*nZ + z)*nY + y)*nX + x                   (Eq. 1.7-1.9)
 *   - U_mu(x) links x to x + mu                                     (Section 1.1)
 *   - Q_munu(x): the four leaves of Eq. 1.12
 *   - self coupling A(x) = (m0 + 4) I_12
 *       - (c_sw/32) sum over all ordered (mu, nu) of
 *         (gamma_mu gamma_nu) (x) (Q_munu(x) - Q_numu(x))            (Eq. 1.11, 2.5)
 *   - (D psi)(x) = A(x) psi(x)
 *       - 1/2 sum_mu ((I_4 - gamma_mu) (x) U_mu(x))       psi(x + mu)
 *       - 1/2 sum_mu ((I_4 + gamma_mu) (x) U_mu^H(x - mu)) psi(x - mu)   (Eq. 1.13, a = 1)
 *
 * Readings where the thesis is silent:
 *   - gamma basis: Euclidean chiral basis, written out below as explicit
 *     4x4 tables (gamma_X,Y,Z = [[0, -i sigma_k], [i sigma_k, 0]] for
 *     k = 1, 2, 3, gamma_T = [[0, I], [I, 0]]).
 *   - boundary: the fermion hop across the T boundary carries the sign
 *     t_bc (-1 antiperiodic, +1 periodic); Z, Y, X are periodic.  Gauge
 *     links are always periodic, so Q_munu carries no sign.
 *
 * Layouts (complex double = interleaved re, im):
 *   psi [V][12], U [V][4][3][3], A [V][12][12], G and F [V][4][3][3].
 */
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <string.h>

typedef double complex cplx;

/* gamma_mu[row][col] for mu = T, Z, Y, X (Euclidean chiral basis). */
static const cplx GAMMA[4][4][4] = {
    /* T */ {{0, 0, 1, 0}, {0, 0, 0, 1}, {1, 0, 0, 0}, {0, 1, 0, 0}},
    /* Z */ {{0, 0, -I, 0}, {0, 0, 0, I}, {I, 0, 0, 0}, {0, -I, 0, 0}},
    /* Y */ {{0, 0, 0, -1}, {0, 0, 1, 0}, {0, 1, 0, 0}, {-1, 0, 0, 0}},
    /* X */ {{0, 0, 0, -I}, {0, 0, -I, 0}, {0, I, 0, 0}, {I, 0, 0, 0}},
};

void oracle_gamma(int mu, cplx out[16]) {
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) out[4 * r + c] = GAMMA[mu][r][c];
}

/* ---- lattice geometry (Eq. 1.7-1.9 and the boundary rule of Section 1.1) ---- */

static int64_t volume(const int d[4]) { return (int64_t)d[0] * d[1] * d[2] * d[3]; }

static void coords(const int d[4], int64_t s, int c[4]) {
  c[3] = (int)(s % d[3]);
  s /= d[3];
  c[2] = (int)(s % d[2]);
  s /= d[2];
  c[1] = (int)(s % d[1]);
  c[0] = (int)(s / d[1]);
}

static int64_t site_of(const int d[4], const int c[4]) {
  return (((int64_t)c[0] * d[1] + c[1]) * d[2] + c[2]) * d[3] + c[3];
}

/* Neighbour x + step*mu (step = +1 or -1) with wrap-around.  *sign receives
 * t_bc when the hop crosses the T boundary, else 1. */
int64_t oracle_shift(const int d[4], int64_t s, int mu, int step, int t_bc, double* sign) {
  int c[4];
  coords(d, s, c);
  int v = c[mu] + step;
  double sg = 1.0;
  if (v >= d[mu]) {
    v -= d[mu];
    if (mu == 0) sg = (double)t_bc;
  } else if (v < 0) {
    v += d[mu];
    if (mu == 0) sg = (double)t_bc;
  }
  c[mu] = v;
  if (sign) *sign = sg;
  return site_of(d, c);
}

/* ---- 3x3 colour matrices ---- */

static const cplx* link(const cplx* U, int64_t s, int mu) { return U + (s * 4 + mu) * 9; }

static void m3_mul(const cplx* A, const cplx* B, cplx* C) {
  cplx t[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      cplx acc = 0;
      for (int k = 0; k < 3; ++k) acc += A[3 * a + k] * B[3 * k + b];
      t[3 * a + b] = acc;
    }
  memcpy(C, t, sizeof t);
}

static void m3_dag(const cplx* A, cplx* B) {
  cplx t[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) t[3 * a + b] = conj(A[3 * b + a]);
  memcpy(B, t, sizeof t);
}

/* ---- Eq. 1.12: the four leaves of Q_munu(x) ----
 * Each leaf is a product of four factors U_{dir}(site) or its conjugate
 * transpose; the list below is the single definition used both to build the
 * clover and to differentiate it. */
typedef struct {
  int64_t site[4];
  int dir[4];
  int dag[4];
} leaf_t;

static void leaves(const int d[4], int64_t x, int mu, int nu, leaf_t L[4]) {
  int64_t xpm = oracle_shift(d, x, mu, +1, 1, 0);
  int64_t xpn = oracle_shift(d, x, nu, +1, 1, 0);
  int64_t xmm = oracle_shift(d, x, mu, -1, 1, 0);
  int64_t xmn = oracle_shift(d, x, nu, -1, 1, 0);
  int64_t xmm_pn = oracle_shift(d, xmm, nu, +1, 1, 0); /* x - mu + nu */
  int64_t xmm_mn = oracle_shift(d, xmm, nu, -1, 1, 0); /* x - mu - nu */
  int64_t xmn_pm = oracle_shift(d, xmn, mu, +1, 1, 0); /* x - nu + mu */
  /* U_mu(x) U_nu(x+mu) U_mu(x+nu)^H U_nu(x)^H */
  L[0] = (leaf_t){{x, xpm, xpn, x}, {mu, nu, mu, nu}, {0, 0, 1, 1}};
  /* U_nu(x) U_mu(x-mu+nu)^H U_nu(x-mu)^H U_mu(x-mu) */
  L[1] = (leaf_t){{x, xmm_pn, xmm, xmm}, {nu, mu, nu, mu}, {0, 1, 1, 0}};
  /* U_mu(x-mu)^H U_nu(x-mu-nu)^H U_mu(x-mu-nu) U_nu(x-nu) */
  L[2] = (leaf_t){{xmm, xmm_mn, xmm_mn, xmn}, {mu, nu, mu, nu}, {1, 1, 0, 0}};
  /* U_nu(x-nu)^H U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^H */
  L[3] = (leaf_t){{xmn, xmn, xmn_pm, x}, {nu, mu, nu, mu}, {1, 0, 0, 1}};
}

static void factor(const cplx* U, const leaf_t* l, int k, cplx F[9]) {
  const cplx* u = link(U, l->site[k], l->dir[k]);
  if (l->dag[k])
    m3_dag(u, F);
  else
    memcpy(F, u, 9 * sizeof(cplx));
}

/* Q_munu(x) per Eq. 1.12. */
void oracle_Q(const int d[4], const cplx* U, int64_t x, int mu, int nu, cplx Q[9]) {
  leaf_t L[4];
  leaves(d, x, mu, nu, L);
  for (int i = 0; i < 9; ++i) Q[i] = 0;
  for (int l = 0; l < 4; ++l) {
    cplx P[9], F[9];
    factor(U, &L[l], 0, P);
    for (int k = 1; k < 4; ++k) {
      factor(U, &L[l], k, F);
      m3_mul(P, F, P);
    }
    for (int i = 0; i < 9; ++i) Q[i] += P[i];
  }
}

/* ---- Eq. 1.11 / 2.5: the 12x12 self coupling A(x) ---- */
void oracle_clover_site(const int d[4], const cplx* U, double m0, double csw, int64_t x, cplx A[144]) {
  for (int i = 0; i < 144; ++i) A[i] = 0;
  for (int i = 0; i < 12; ++i) A[13 * i] = m0 + 4.0;
  for (int mu = 0; mu < 4; ++mu)
    for (int nu = 0; nu < 4; ++nu) {
      cplx Qmn[9], Qnm[9], F[9], GG[16];
      oracle_Q(d, U, x, mu, nu, Qmn);
      oracle_Q(d, U, x, nu, mu, Qnm);
      for (int i = 0; i < 9; ++i) F[i] = Qmn[i] - Qnm[i];
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
          cplx acc = 0;
          for (int k = 0; k < 4; ++k) acc += GAMMA[mu][r][k] * GAMMA[nu][k][c];
          GG[4 * r + c] = acc;
        }
      /* (gamma_mu gamma_nu) (x) F: entry (3 s + a, 3 s' + b) = GG[s][s'] F[a][b] */
      for (int s = 0; s < 4; ++s)
        for (int sp = 0; sp < 4; ++sp)
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
              A[(3 * s + a) * 12 + 3 * sp + b] -= (csw / 32.0) * GG[4 * s + sp] * F[3 * a + b];
    }
}

/* A(x) for a list of sites: A[i] = A(sites[i]). */
void oracle_clover_sites(const int d[4], const cplx* U, double m0, double csw, const int64_t* sites, int64_t n,
                         cplx* A) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) oracle_clover_site(d, U, m0, csw, sites[i], A + i * 144);
}

/* Threads an OpenMP loop of this library uses. */
int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Set the threads of later OpenMP loops (n >= 1), for timing the oracle on one
 * core beside all cores; no effect on the arithmetic. */
void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

void oracle_clover_field(const int d[4], const cplx* U, double m0, double csw, cplx* A) {
  const int64_t V = volume(d);
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < V; ++x) oracle_clover_site(d, U, m0, csw, x, A + x * 144);
}

/* ---- Eq. 1.13 ---- */

/* out += coef * ((P (x) W) in), P a 4x4 spin matrix, W a 3x3 colour matrix. */
static void kron_apply(const cplx P[4][4], const cplx* W, const cplx* in, cplx coef, cplx* out) {
  for (int s = 0; s < 4; ++s)
    for (int a = 0; a < 3; ++a) {
      cplx acc = 0;
      for (int sp = 0; sp < 4; ++sp)
        for (int b = 0; b < 3; ++b) acc += P[s][sp] * W[3 * a + b] * in[3 * sp + b];
      out[3 * s + a] += coef * acc;
    }
}

/* I_4 + sgn * gamma_mu */
static void one_plus(int mu, double sgn, cplx P[4][4]) {
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) P[r][c] = (r == c ? 1.0 : 0.0) + sgn * GAMMA[mu][r][c];
}

/* (D psi)(x) for one site; A_x is that site's 12x12 self coupling. */
void oracle_D_site(const int d[4], int t_bc, const cplx* U, const cplx* A_x, const cplx* psi, int64_t x,
                   cplx out[12]) {
  for (int i = 0; i < 12; ++i) {
    cplx acc = 0;
    for (int j = 0; j < 12; ++j) acc += A_x[12 * i + j] * psi[x * 12 + j];
    out[i] = acc;
  }
  for (int mu = 0; mu < 4; ++mu) {
    cplx P[4][4], W[9];
    double sg;
    /* - 1/2 ((I - gamma_mu) (x) U_mu(x)) psi(x + mu) */
    int64_t y = oracle_shift(d, x, mu, +1, t_bc, &sg);
    one_plus(mu, -1.0, P);
    kron_apply(P, link(U, x, mu), psi + y * 12, -0.5 * sg, out);
    /* - 1/2 ((I + gamma_mu) (x) U_mu^H(x - mu)) psi(x - mu) */
    y = oracle_shift(d, x, mu, -1, t_bc, &sg);
    one_plus(mu, +1.0, P);
    m3_dag(link(U, y, mu), W);
    kron_apply(P, W, psi + y * 12, -0.5 * sg, out);
  }
}

void oracle_apply_D(const int d[4], int t_bc, const cplx* U, const cplx* A, const cplx* psi, cplx* out) {
  const int64_t V = volume(d);
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < V; ++x) oracle_D_site(d, t_bc, U, A + x * 144, psi, x, out + x * 12);
}

/* (D psi) at a list of sites only; A holds the self coupling of those sites
 * in the same order ([nsites][144]). */
void oracle_apply_D_sites(const int d[4], int t_bc, const cplx* U, const cplx* A, const cplx* psi,
                          const int64_t* sites, int64_t nsites, cplx* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < nsites; ++i) oracle_D_site(d, t_bc, U, A + i * 144, psi, sites[i], out + i * 12);
}

/* D^H as the conjugate transpose of the term list of Eq. 1.13: every term
 * "out(x) += M in(y)" of D becomes "out(y) += M^H in(x)".  Serial on purpose
 * (a scatter). */
void oracle_apply_DH(const int d[4], int t_bc, const cplx* U, const cplx* A, const cplx* psi, cplx* out) {
  const int64_t V = volume(d);
  memset(out, 0, (size_t)V * 12 * sizeof(cplx));
  for (int64_t x = 0; x < V; ++x) {
    const cplx* Ax = A + x * 144;
    for (int i = 0; i < 12; ++i) { /* A(x)^H psi(x) */
      cplx acc = 0;
      for (int j = 0; j < 12; ++j) acc += conj(Ax[12 * j + i]) * psi[x * 12 + j];
      out[x * 12 + i] += acc;
    }
    for (int mu = 0; mu < 4; ++mu) {
      cplx P[4][4], PH[4][4], W[9];
      double sg;
      /* term of D: out(x) += -1/2 sg ((I - g) (x) U_mu(x)) in(x+mu); adjoint:
         out(x+mu) += -1/2 sg ((I - g)^H (x) U_mu(x)^H) in(x) */
      int64_t y = oracle_shift(d, x, mu, +1, t_bc, &sg);
      one_plus(mu, -1.0, P);
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) PH[r][c] = conj(P[c][r]);
      m3_dag(link(U, x, mu), W);
      kron_apply((const cplx(*)[4])PH, W, psi + x * 12, -0.5 * sg, out + y * 12);
      /* term of D: out(x) += -1/2 sg ((I + g) (x) U_mu(x-mu)^H) in(x-mu); adjoint:
         out(x-mu) += -1/2 sg ((I + g)^H (x) U_mu(x-mu)) in(x) */
      y = oracle_shift(d, x, mu, -1, t_bc, &sg);
      one_plus(mu, +1.0, P);
      for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) PH[r][c] = conj(P[c][r]);
      kron_apply((const cplx(*)[4])PH, link(U, y, mu), psi + x * 12, -0.5 * sg, out + y * 12);
    }
  }
}

/* ---- derivative of L = Re <phi, D psi> = Re sum_x phi(x)^H (D psi)(x) ----
 * G_mu(x) = dL/dRe U_mu(x) + i dL/dIm U_mu(x) (the convention of torch's
 * complex gradients), so that dL = Re tr(G^H dU).
 * L depends on a link U through terms Re tr(U R) (G += R^H) and
 * Re tr(U^H R) (G += R). */

static void add_dag(cplx* G, const cplx* R) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) G[3 * a + b] += conj(R[3 * b + a]);
}

/* Hopping part of Eq. 1.13 (self coupling held fixed). */
void oracle_force_hop(const int d[4], int t_bc, const cplx* U, const cplx* phi, const cplx* psi, cplx* G) {
  const int64_t V = volume(d);
#pragma omp parallel for schedule(static)
  for (int64_t x = 0; x < V; ++x)
    for (int mu = 0; mu < 4; ++mu) {
      cplx* g = G + (x * 4 + mu) * 9;
      double sg;
      int64_t y = oracle_shift(d, x, mu, +1, t_bc, &sg);
      cplx Pm[4][4], Pp[4][4];
      one_plus(mu, -1.0, Pm);
      one_plus(mu, +1.0, Pp);
      /* forward term at output x: -1/2 sg phi(x)^H ((I - g) (x) U) psi(y) = tr(U R1),
         R1[b][a] = -1/2 sg sum_{s,s'} (I - g)[s][s'] psi(y)[s'][b] conj(phi(x)[s][a]) */
      cplx R1[9], R2[9];
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
          cplx acc = 0;
          for (int s = 0; s < 4; ++s)
            for (int sp = 0; sp < 4; ++sp)
              acc += Pm[s][sp] * psi[y * 12 + 3 * sp + b] * conj(phi[x * 12 + 3 * s + a]);
          R1[3 * b + a] = -0.5 * sg * acc;
        }
      /* backward term at output y: -1/2 sg phi(y)^H ((I + g) (x) U^H) psi(x)
         = sum_{a,b} conj(U[b][a]) X[a][b] = tr(U^H R2) with R2[b][a] = X[a][b],
         X[a][b] = -1/2 sg sum_{s,s'} (I + g)[s][s'] psi(x)[s'][b] conj(phi(y)[s][a]) */
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          cplx acc = 0;
          for (int s = 0; s < 4; ++s)
            for (int sp = 0; sp < 4; ++sp)
              acc += Pp[s][sp] * psi[x * 12 + 3 * sp + b] * conj(phi[y * 12 + 3 * s + a]);
          R2[3 * b + a] = -0.5 * sg * acc;
        }
      for (int i = 0; i < 9; ++i) g[i] = 0;
      add_dag(g, R1);
      for (int i = 0; i < 9; ++i) g[i] += R2[i];
    }
}

/* Self-coupling part: L_sc = Re sum_x phi(x)^H A(x) psi(x) with A(x) built
 * from the links (Eq. 1.11, 1.12).  Only the field-strength term depends on
 * U:  L_sc = const + Re sum_x sum_{mu,nu} tr((Q_munu(x) - Q_numu(x)) T_munu(x)),
 * T_munu[b][a] = -(c_sw/32) sum_{s,s'} (gamma_mu gamma_nu)[s][s'] psi(x)[s'][b] conj(phi(x)[s][a]).
 * For a leaf F1 F2 F3 F4, tr(F1 F2 F3 F4 T) = tr(F_k R) with
 * R = F_{k+1} .. F4 T F1 .. F_{k-1}.  Accumulated serially (a scatter). */
void oracle_force_clover(const int d[4], const cplx* U, double csw, const cplx* phi, const cplx* psi, cplx* G) {
  const int64_t V = volume(d);
  for (int64_t x = 0; x < V; ++x)
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = 0; nu < 4; ++nu) {
        if (mu == nu) continue; /* Q_mumu - Q_mumu = 0 */
        cplx GG[4][4], T[9];
        for (int r = 0; r < 4; ++r)
          for (int c = 0; c < 4; ++c) {
            cplx acc = 0;
            for (int k = 0; k < 4; ++k) acc += GAMMA[mu][r][k] * GAMMA[nu][k][c];
            GG[r][c] = acc;
          }
        for (int b = 0; b < 3; ++b)
          for (int a = 0; a < 3; ++a) {
            cplx acc = 0;
            for (int s = 0; s < 4; ++s)
              for (int sp = 0; sp < 4; ++sp) acc += GG[s][sp] * psi[x * 12 + 3 * sp + b] * conj(phi[x * 12 + 3 * s + a]);
            T[3 * b + a] = -(csw / 32.0) * acc;
          }
        /* +Q_munu(x) and -Q_numu(x) */
        for (int pass = 0; pass < 2; ++pass) {
          leaf_t L[4];
          double w = pass == 0 ? 1.0 : -1.0;
          if (pass == 0)
            leaves(d, x, mu, nu, L);
          else
            leaves(d, x, nu, mu, L);
          for (int l = 0; l < 4; ++l)
            for (int k = 0; k < 4; ++k) {
              cplx R[9], F[9];
              /* R = F_{k+1} .. F_4 T F_1 .. F_{k-1} */
              for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
              for (int j = k + 1; j < 4; ++j) {
                factor(U, &L[l], j, F);
                m3_mul(R, F, R);
              }
              m3_mul(R, T, R);
              for (int j = 0; j < k; ++j) {
                factor(U, &L[l], j, F);
                m3_mul(R, F, R);
              }
              cplx* g = G + (L[l].site[k] * 4 + L[l].dir[k]) * 9;
              if (L[l].dag[k]) { /* tr(U^H R): G += R */
                for (int i = 0; i < 9; ++i) g[i] += w * R[i];
              } else { /* tr(U R): G += R^H */
                cplx Rw[9];
                for (int i = 0; i < 9; ++i) Rw[i] = w * R[i];
                add_dag(g, Rw);
              }
            }
        }
      }
}

/* F = P(G U^H), P(M) = (M - M^H)/2 - tr(M - M^H)/6 I: the su(3) component
 * such that d/de L(exp(e X) U) at e = 0 equals Re tr(F^H X) for X in su(3). */
void oracle_force_project(int64_t nlinks, const cplx* U, const cplx* G, cplx* F) {
#pragma omp parallel for schedule(static)
  for (int64_t l = 0; l < nlinks; ++l) {
    cplx Ud[9], M[9];
    m3_dag(U + l * 9, Ud);
    m3_mul(G + l * 9, Ud, M);
    cplx* f = F + l * 9;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) f[3 * a + b] = 0.5 * (M[3 * a + b] - conj(M[3 * b + a]));
    cplx tr = (f[0] + f[4] + f[8]) / 3.0;
    for (int a = 0; a < 3; ++a) f[4 * a] -= tr;
  }
}
